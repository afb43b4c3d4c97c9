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
           "ob_price_ask_bid_noalloc")


class ObStats(ctypes.Structure):
    _fields_ = [("options", ctypes.c_int64), ("node_updates", ctypes.c_int64),
                ("u_points", ctypes.c_int64), ("w_points", ctypes.c_int64),
                ("z_points", ctypes.c_int64),
                ("max_level_points", ctypes.c_int32), ("retried", ctypes.c_int32),
                ("failed", ctypes.c_int32), ("tiers", ctypes.c_int32)]


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
                     "ob_price_ask_bid_noalloc"):
            f = getattr(lib, name)
            f.argtypes = [P, i64, P, P, P]
            f.restype = ctypes.c_int
        lib.ob_price_ask_bid_host.argtypes = [P, i64, P, P]
        lib.ob_price_ask_bid_host.restype = ctypes.c_int
        lib.ob_get_stats.argtypes = [ctypes.POINTER(ObStats)]
        lib.ob_get_stats.restype = ctypes.c_int
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


def ob_price_ask_bid_plain(params, n, out, status=None, stream=None):
    _check(load().ob_price_ask_bid_plain(_ptr(params), int(n), _ptr(out), _ptr(status),
                                         _stream(stream)))


def ob_crr_american(params, n, out, status=None, stream=None):
    _check(load().ob_crr_american(_ptr(params), int(n), _ptr(out), _ptr(status), _stream(stream)))


def ob_price_ask_bid_noalloc(params, n, out, status=None, stream=None):
    """Fixed-scratch form: for callers that cannot allocate device memory when they price
    (the library's pool is never touched; scratch is a device array held since load time).
    At most 4096 options per call; calls that overlap on the GPU must be serialised."""
    _check(load().ob_price_ask_bid_noalloc(_ptr(params), int(n), _ptr(out), _ptr(status),
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


def ob_release():
    _check(load().ob_release())


# ---------------------------------------------------------------- conveniences
def price(table, plain=False, stream=None):
    """ask/bid of a workloads table on the current CUDA device: (out[n,2], status[n]) tensors."""
    import torch
    n = int(np.asarray(table).shape[0])
    dev = to_device(table)
    out = torch.empty((n, 2), dtype=torch.float64, device=dev.device)
    st = torch.empty(n, dtype=torch.int32, device=dev.device)
    (ob_price_ask_bid_plain if plain else ob_price_ask_bid)(dev, n, out, st, stream)
    return out, st


def crr(table, stream=None):
    import torch
    n = int(np.asarray(table).shape[0])
    dev = to_device(table)
    out = torch.empty(n, dtype=torch.float64, device=dev.device)
    st = torch.empty(n, dtype=torch.int32, device=dev.device)
    ob_crr_american(dev, n, out, st, stream)
    return out, st
