"""Python binding of the GB300 ask/bid pricer (libob.so, C ABI in include/ob.h).

Argument marshalling only: device memory and streams come from PyTorch, every
step of the pricing runs in the library's CUDA kernels.  There is no CPU path:
if libob.so is missing or no CUDA device is present the calls raise.

Entry points (same names as the C ABI):
  ob_price_ask_bid(params, n, out, status, stream)        batched, work-stealing
  ob_price_ask_bid_plain(params, n, out, status, stream)  one warp per option
  ob_crr_american(params, n, out, status, stream)         plain CRR, no costs
  ob_price_ask_bid_host(params_np, out_np, status_np)     host buffers, synchronous
  ob_get_stats(), ob_release(), ob_strerror(code)
plus small helpers to move a workloads table to the device.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libob.so")
_lib = None

OB_OK, OB_ERR_ARG, OB_ERR_ARBITRAGE, OB_ERR_CAPACITY, OB_ERR_TIMEOUT, OB_ERR_CUDA, OB_ERR_NOMEM = (
    0, -1, -2, -3, -4, -5, -6)

EXPORTS = ("ob_price_ask_bid", "ob_price_ask_bid_plain", "ob_crr_american", "ob_price_ask_bid_host",
           "ob_get_stats", "ob_release", "ob_strerror", "ob_last_cuda_error",
           "ob_price_ask_bid_noalloc", "ob_greeks", "ob_configure", "ob_autotune",
           "ob_price_ask_bid_wide", "ob_fp64_peak", "ob_crr_american_wide", "ob_price_ask_bid_hedge",
           "ob_hedge_path")


class ObStats(ctypes.Structure):
    _fields_ = [("options", ctypes.c_int64), ("node_updates", ctypes.c_int64),
                ("u_points", ctypes.c_int64), ("w_points", ctypes.c_int64),
                ("z_points", ctypes.c_int64),
                ("max_level_points", ctypes.c_int32), ("retried", ctypes.c_int32),
                ("failed", ctypes.c_int32), ("tiers", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("team_warps", ctypes.c_int32),
                ("chip_points", ctypes.c_int32), ("half_teams", ctypes.c_int32)]


class ObError(RuntimeError):
    pass


def load():
    """Load libob.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ObError("libob.so not built: run __graft_entry__.build() (no CPU fallback exists)")
        lib = ctypes.CDLL(LIB_PATH)
        P, i64 = ctypes.c_void_p, ctypes.c_int64
        for name in ("ob_price_ask_bid", "ob_price_ask_bid_plain", "ob_crr_american",
                     "ob_price_ask_bid_noalloc", "ob_greeks", "ob_price_ask_bid_wide",
                     "ob_crr_american_wide"):
            f = getattr(lib, name)
            f.argtypes = [P, i64, P, P, P]
            f.restype = ctypes.c_int
        lib.ob_greeks.argtypes = [P, i64, P, P, P, P]
        lib.ob_greeks.restype = ctypes.c_int
        lib.ob_price_ask_bid_hedge.argtypes = [P, i64, P, P, P, P]
        lib.ob_price_ask_bid_hedge.restype = ctypes.c_int
        lib.ob_hedge_path.argtypes = [P, i64, P, i64, P, P, P, P, P, P]
        lib.ob_hedge_path.restype = ctypes.c_int
        lib.ob_price_ask_bid_host.argtypes = [P, i64, P, P]
        lib.ob_price_ask_bid_host.restype = ctypes.c_int
        lib.ob_get_stats.argtypes = [ctypes.POINTER(ObStats)]
        lib.ob_get_stats.restype = ctypes.c_int
        lib.ob_configure.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        lib.ob_configure.restype = ctypes.c_int
        lib.ob_autotune.argtypes = [P, i64, i64, P, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)]
        lib.ob_autotune.restype = ctypes.c_int
        lib.ob_fp64_peak.argtypes = [i64, P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.ob_fp64_peak.restype = ctypes.c_int
        lib.ob_release.argtypes = []
        lib.ob_release.restype = ctypes.c_int
        lib.ob_strerror.argtypes = [ctypes.c_int]
        lib.ob_strerror.restype = ctypes.c_char_p
        lib.ob_last_cuda_error.argtypes = []
        lib.ob_last_cuda_error.restype = ctypes.c_char_p
        _lib = lib
    return _lib


def ob_strerror(code: int) -> str:
    return load().ob_strerror(int(code)).decode()


def _check(rc: int):
    if rc != OB_OK:
        msg = ob_strerror(rc)
        if rc == OB_ERR_CUDA:
            msg += ": " + load().ob_last_cuda_error().decode()
        raise ObError("libob: %s (%d)" % (msg, rc))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def to_device(table, device="cuda"):
    """A workloads table (numpy structured array, 64-byte records) as a uint8 CUDA tensor."""
    import torch
    a = np.ascontiguousarray(table)
    if a.dtype.itemsize != 64:
        raise ValueError("records must be 64 bytes")
    return torch.from_numpy(a.view(np.uint8).reshape(-1).copy()).to(device)


def ob_price_ask_bid(params, n, out, status=None, stream=None):
    _check(load().ob_price_ask_bid(_ptr(params), int(n), _ptr(out), _ptr(status), _stream(stream)))


def ob_price_ask_bid_hedge(params, n, out, status, hedge, stream=None):
    """ob_price_ask_bid plus the hedge at the root: hedge[n, 4] = (seller's stock holding after
    rebalancing at t = 0, buyer's, immediate exercise sets the ask, buyer exercises at once)."""
    _check(load().ob_price_ask_bid_hedge(_ptr(params), int(n), _ptr(out), _ptr(status), _ptr(hedge),
                                         _stream(stream)))


def ob_hedge_path(params, n, moves, stride, out, hold, cash, stop, status=None, stream=None):
    """The hedge along one path per option: moves[n, stride] int8 (non-zero up), out[n, 2] ask/bid,
    hold[n, stride + 1, 2] the seller's and buyer's holdings after rebalancing at each level,
    cash (same shape, or None) their cash after rebalancing, stop[n] the buyer's stopping level
    (-1: never)."""
    _check(load().ob_hedge_path(_ptr(params), int(n), _ptr(moves), int(stride), _ptr(out), _ptr(hold),
                                _ptr(cash), _ptr(stop), _ptr(status), _stream(stream)))


def ob_price_ask_bid_plain(params, n, out, status=None, stream=None):
    _check(load().ob_price_ask_bid_plain(_ptr(params), int(n), _ptr(out), _ptr(status),
                                         _stream(stream)))


def ob_price_ask_bid_wide(params, n, out, status=None, stream=None):
    """Whole-GPU form: each option in turn on every SM (large single options)."""
    _check(load().ob_price_ask_bid_wide(_ptr(params), int(n), _ptr(out), _ptr(status),
                                        _stream(stream)))


def ob_crr_american(params, n, out, status=None, stream=None):
    _check(load().ob_crr_american(_ptr(params), int(n), _ptr(out), _ptr(status), _stream(stream)))


def ob_crr_american_wide(params, n, out, status=None, stream=None):
    """Whole-GPU CRR form: each option in turn on every SM (large single options)."""
    _check(load().ob_crr_american_wide(_ptr(params), int(n), _ptr(out), _ptr(status), _stream(stream)))


def ob_price_ask_bid_noalloc(params, n, out, status=None, stream=None):
    """Fixed-scratch form: for callers that cannot allocate device memory when they price
    (the library's pool is never touched; scratch is a device array held since load time).
    At most 4096 options per call; calls that overlap on the GPU must be serialised."""
    _check(load().ob_price_ask_bid_noalloc(_ptr(params), int(n), _ptr(out), _ptr(status),
                                           _stream(stream)))


def ob_greeks(params, n, out, grad, status=None, stream=None):
    """Prices and d(ask, bid)/d(S0, K, sigma, R, T, k): out (n x 2), grad (n x 2 x 6), device tensors."""
    _check(load().ob_greeks(_ptr(params), int(n), _ptr(out), _ptr(grad), _ptr(status),
                            _stream(stream)))


def ob_price_ask_bid_host(params, out, status=None):
    """Host buffers: params (numpy records), out (n x 2 float64), status (n int32) or None."""
    a = np.ascontiguousarray(params)
    assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == 2 * a.shape[0]
    st = None if status is None else status.ctypes.data_as(ctypes.c_void_p)
    _check(load().ob_price_ask_bid_host(a.ctypes.data_as(ctypes.c_void_p), a.shape[0],
                                        out.ctypes.data_as(ctypes.c_void_p), st))


def ob_get_stats() -> dict:
    s = ObStats()
    _check(load().ob_get_stats(ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in ObStats._fields_}


def ob_fp64_peak(iters=1 << 16, stream=None):
    """Measured FP64 FMA throughput of the device: (TFLOP/s, ms of the timed launch)."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().ob_fp64_peak(int(iters), _stream(stream), ctypes.byref(tf), ctypes.byref(ms)))
    return float(tf.value), float(ms.value)


def ob_release():
    _check(load().ob_release())


def ob_configure(team_warps=0, use_graphs=-1, chip_points=-2):
    """Team width of the batched form (4, 8, 12, 16; 0 keeps), CUDA-graph replay (1, 0; -1 keeps)
    and the on-chip w points of the fused level step (-1 all that fit, 0 off, -2 keeps)."""
    _check(load().ob_configure(int(team_warps), int(use_graphs), int(chip_points)))


TUNE_CANDIDATES = ("16", "16-whole", "12", "8", "4", "16+chip", "8+chip")


def ob_autotune(params, n, sample=0, stream=None):
    """Time the seven configurations of TUNE_CANDIDATES on a sample of the device records and
    keep the fastest ("16": 16-warp teams that split into two 8-warp teams for the light
    options; "16-whole": no split).  Returns (team_warps, chip_points, {candidate: ms})."""
    tw = ctypes.c_int32(0)
    chip = ctypes.c_int32(0)
    ms = (ctypes.c_float * len(TUNE_CANDIDATES))()
    _check(load().ob_autotune(_ptr(params), int(n), int(sample), _stream(stream), ctypes.byref(tw),
                              ctypes.byref(chip), ms))
    return int(tw.value), int(chip.value), {k: float(v) for k, v in zip(TUNE_CANDIDATES, ms)}


def autotune(table, sample=0):
    """ob_autotune on a workloads table: (team_warps, chip_points, {candidate: ms})."""
    dev = to_device(table)
    return ob_autotune(dev, int(np.asarray(table).shape[0]), sample)


# ---------------------------------------------------------------- conveniences
def price(table, plain=False, stream=None, wide=False):
    """ask/bid of a workloads table on the current CUDA device: (out[n,2], status[n]) tensors.
    plain: one warp per option; wide: each option on the whole GPU; else the batched form."""
    import torch
    n = int(np.asarray(table).shape[0])
    dev = to_device(table)
    out = torch.empty((n, 2), dtype=torch.float64, device=dev.device)
    st = torch.empty(n, dtype=torch.int32, device=dev.device)
    f = ob_price_ask_bid_wide if wide else (ob_price_ask_bid_plain if plain else ob_price_ask_bid)
    f(dev, n, out, st, stream)
    return out, st


def hedge(table, stream=None):
    """ask/bid and the hedge at the root of a workloads table: (out[n,2], hedge[n,4], status[n])."""
    import torch
    n = int(np.asarray(table).shape[0])
    dev = to_device(table)
    out = torch.empty((n, 2), dtype=torch.float64, device=dev.device)
    hg = torch.empty((n, 4), dtype=torch.float64, device=dev.device)
    st = torch.empty(n, dtype=torch.int32, device=dev.device)
    ob_price_ask_bid_hedge(dev, n, out, st, hg, stream)
    return out, hg, st


def hedge_path(table, moves, stream=None):
    """The hedge along the paths moves[n, stride] (int8, non-zero up) of a workloads table:
    (out[n,2], hold[n,stride+1,2], cash[n,stride+1,2], stop[n], status[n]) tensors."""
    import torch
    n = int(np.asarray(table).shape[0])
    dev = to_device(table)
    mv = torch.as_tensor(np.ascontiguousarray(moves, dtype=np.int8)).to(dev.device)
    if mv.dim() != 2 or mv.shape[0] != n:
        raise ValueError("moves must be [n_options, stride]")
    stride = max(int(mv.shape[1]), 1)
    if mv.shape[1] == 0:
        mv = torch.zeros((n, 1), dtype=torch.int8, device=dev.device)
    out = torch.empty((n, 2), dtype=torch.float64, device=dev.device)
    hold = torch.empty((n, stride + 1, 2), dtype=torch.float64, device=dev.device)
    cash = torch.empty_like(hold)
    stop = torch.empty(n, dtype=torch.int32, device=dev.device)
    st = torch.empty(n, dtype=torch.int32, device=dev.device)
    ob_hedge_path(dev, n, mv, stride, out, hold, cash, stop, st, stream)
    return out, hold, cash, stop, st


def crr(table, stream=None, wide=False):
    """Plain CRR prices of a workloads table: (out[n], status[n]) tensors; wide: each option
    on the whole GPU."""
    import torch
    n = int(np.asarray(table).shape[0])
    dev = to_device(table)
    out = torch.empty(n, dtype=torch.float64, device=dev.device)
    st = torch.empty(n, dtype=torch.int32, device=dev.device)
    (ob_crr_american_wide if wide else ob_crr_american)(dev, n, out, st, stream)
    return out, st


def greeks(table, stream=None):
    """Prices and gradients of a workloads table: (out[n,2], grad[n,2,6], status[n]) tensors."""
    import torch
    n = int(np.asarray(table).shape[0])
    dev = to_device(table)
    out = torch.empty((n, 2), dtype=torch.float64, device=dev.device)
    grad = torch.empty((n, 2, 6), dtype=torch.float64, device=dev.device)
    st = torch.empty(n, dtype=torch.int32, device=dev.device)
    ob_greeks(dev, n, out, grad, st, stream)
    return out, grad, st


def pack_params(theta, width, N, payoff):
    """64-byte option records from tensors: theta (n, 6) float64 = (S0, K, sigma, R, T, k),
    width (n,) = K2 - K, N and payoff (n,) int32.  Plain tensor marshalling."""
    import torch
    S0, K, sig, R, T, k = theta.unbind(1)
    d = torch.stack([S0, K, K + width, sig, R, T, k], dim=1)
    ints = torch.stack([N.to(torch.int32), payoff.to(torch.int32)], dim=1).contiguous()
    rec = torch.cat([d, ints.view(torch.float64)], dim=1).contiguous()
    return rec.view(torch.uint8).reshape(-1)


def _autograd_class():
    import torch

    class AskBid(torch.autograd.Function):
        """(ask, bid) of American options with proportional costs as a differentiable function
        of theta = (S0, K, sigma, R, T, k).  The forward calls ob_greeks (prices and the adjoint
        in one launch); the backward contracts the stored gradient with the incoming ones."""

        @staticmethod
        def forward(ctx, theta, width, N, payoff):
            n = theta.shape[0]
            params = pack_params(theta.detach(), width, N, payoff)
            out = torch.empty((n, 2), dtype=torch.float64, device=theta.device)
            grad = torch.empty((n, 2, 6), dtype=torch.float64, device=theta.device)
            st = torch.empty(n, dtype=torch.int32, device=theta.device)
            ob_greeks(params, n, out, grad, st)
            ctx.save_for_backward(grad)
            ctx.mark_non_differentiable(st)
            return out[:, 0].clone(), out[:, 1].clone(), st

        @staticmethod
        def backward(ctx, g_ask, g_bid, g_st):
            (grad,) = ctx.saved_tensors
            g = torch.zeros_like(grad[:, 0, :])
            if g_ask is not None:
                g = g + g_ask[:, None] * grad[:, 0, :]
            if g_bid is not None:
                g = g + g_bid[:, None] * grad[:, 1, :]
            return g, None, None, None

    return AskBid


_AskBid = None


def ask_bid(theta, width, N, payoff):
    """Differentiable (ask, bid, status): see AskBid."""
    global _AskBid
    if _AskBid is None:
        _AskBid = _autograd_class()
    return _AskBid.apply(theta, width, N, payoff)
