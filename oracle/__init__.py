"""CPU oracle -- TEST INFRASTRUCTURE, not part of the product path.

A slow, independent FP64 reference for the ask/bid induction of Zhang, Roux
and Zastawniak (Section 3 and Section 4.1; the sequential procedures are
Roux & Zastawniak's Algorithms 3.1 and 3.5), for the plain CRR recursion
(Section 3 first paragraph and the Appendix) and for the derivatives of ask
and bid by forward-mode dual numbers.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: the C++ source here (``ob_oracle.cpp``) is compiled by ``gcc`` into
``liboboracle.so`` and loaded with ctypes.

``alg1_price`` runs the paper's own parallel scheme (Section 4.2, Algorithm 1: blocks of
levels split into regions A and B, signals between neighbouring threads, a barrier per
round, fewer threads near the root) over the same node steps, as a CPU comparator.

Sub-modules:
  * ``exact``      -- the same recursion in exact rational arithmetic.
  * ``hedging_lp`` -- brute-force superhedging / stopping-time linear programs
                      on the non-recombining tree (an independent formulation).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ob_oracle.cpp")
_LIB = os.path.join(_HERE, "liboboracle.so")
_lock = threading.Lock()
_lib = None

# Error codes of the oracle (its own numbering).
OK, ERR_ARG, ERR_ARBITRAGE, ERR_UNBOUNDED, ERR_CAPACITY = 0, -1, -2, -3, -4
PUT, CALL, SPREAD = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ``ob_oracle.cpp`` into ``liboboracle.so`` (plain g++, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-shared", "-fPIC",
               "-pthread", _SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int
            d = ctypes.c_double
            lib.or_price_tc.argtypes = [P, i64, P, P, i32]
            lib.or_tc_stats.argtypes = [P, P, P]
            lib.or_greeks_tc.argtypes = [P, i64, P, P, P, i32]
            lib.or_price_crr.argtypes = [P, i64, P, P, i32, i32]
            lib.or_pl_envelope.argtypes = [P, P, i32, d, d, P, P, i32, d, d, i32, P, P, i32, P, P]
            lib.or_pl_restrict.argtypes = [P, P, i32, d, d, d, d, P, P, i32, P, P]
            lib.or_pl_eval.argtypes = [P, P, i32, d, d, P, i32, P]
            lib.or_node_step.argtypes = [P, P, i32, d, d, P, P, i32, d, d, d, d, d, d, d, i32,
                                         P, P, i32, P, P]
            lib.or_initial_hedge.argtypes = [P, i64, P, P, i32]
            lib.or_pl_rebalance.argtypes = [P, P, i32, d, d, d, d, d, P, P]
            lib.or_root_objective.argtypes = [P, i32, P, i32, P]
            lib.or_hedge_path.argtypes = [P, i64, P, i64, P, P, P, P, i32]
            lib.or_alg1_tc.argtypes = [P, i32, i32, P, P, P]
            lib.or_alg1_crr.argtypes = [P, i32, i32, P, P, P]
            lib.or_alg1_rounds.argtypes = [i32, i32, i32, P, i32]
            for f in (lib.or_price_tc, lib.or_tc_stats, lib.or_greeks_tc, lib.or_price_crr,
                      lib.or_pl_envelope, lib.or_pl_restrict, lib.or_pl_eval, lib.or_node_step,
                      lib.or_alg1_tc, lib.or_alg1_crr, lib.or_alg1_rounds, lib.or_initial_hedge,
                      lib.or_pl_rebalance, lib.or_root_objective, lib.or_hedge_path):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _as_table(opts) -> np.ndarray:
    from workloads import OPTION_DTYPE  # seeded generators / record layout only
    a = np.ascontiguousarray(opts)
    if a.dtype != OPTION_DTYPE:
        raise TypeError("option table must have dtype workloads.OPTION_DTYPE")
    return a.reshape(-1)


def _threads(nthreads):
    return int(nthreads) if nthreads else 1


def price_ask_bid(opts, nthreads: int = 1):
    """ask/bid of each option: returns (out[n, 2], status[n])."""
    a = _as_table(opts)
    n = a.shape[0]
    out = np.empty((n, 2), np.float64)
    st = np.empty(n, np.int32)
    _load().or_price_tc(_ptr(a), n, _ptr(out), _ptr(st), _threads(nthreads))
    return out, st


def greeks(opts, nthreads: int = 1):
    """(out[n,2], grad[n,2,6], status[n]); grad[i,0] = d ask / d(S0,K,sigma,R,T,k), grad[i,1] for bid."""
    a = _as_table(opts)
    n = a.shape[0]
    out = np.empty((n, 2), np.float64)
    grad = np.empty((n, 2, 6), np.float64)
    st = np.empty(n, np.int32)
    _load().or_greeks_tc(_ptr(a), n, _ptr(out), _ptr(grad), _ptr(st), _threads(nthreads))
    return out, grad, st


def crr_price(opts, american: bool = True, nthreads: int = 1):
    """Plain CRR price without costs (European when american=False): (out[n], status[n])."""
    a = _as_table(opts)
    n = a.shape[0]
    out = np.empty(n, np.float64)
    st = np.empty(n, np.int32)
    _load().or_price_crr(_ptr(a), n, _ptr(out), _ptr(st), 1 if american else 0, _threads(nthreads))
    return out, st


def tc_stats(opt):
    """Breakpoint statistics of one option: dict with nodes, sums, maxima and per-level sums."""
    a = _as_table(opt)[:1]
    N = int(a["N"][0])
    counts = np.zeros(5, np.int64)
    per = np.zeros(2 * (N + 1), np.int64)
    rc = _load().or_tc_stats(_ptr(a), _ptr(counts), _ptr(per))
    if rc:
        raise ValueError("oracle error %d" % rc)
    return {"nodes": int(counts[0]), "bp_seller": int(counts[1]), "bp_buyer": int(counts[2]),
            "max_seller": int(counts[3]), "max_buyer": int(counts[4]),
            "per_level_seller": per[0::2].copy(), "per_level_buyer": per[1::2].copy()}


def initial_hedge(opts, nthreads: int = 1):
    """The hedge at the root (Section 3's rebalancing at t = 0): out[n, 4] = (seller's stock
    holding y*, buyer's y*, 1 if immediate exercise sets the ask, 1 if the buyer exercises at
    once), status[n]."""
    a = _as_table(opts)
    n = a.shape[0]
    out = np.empty((n, 4), np.float64)
    st = np.empty(n, np.int32)
    _load().or_initial_hedge(_ptr(a), n, _ptr(out), _ptr(st), _threads(nthreads))
    return out, st


def hedge_path(opts, moves, nthreads: int = 1):
    """The hedge along a path of each option: moves[n, stride] (1 up, 0 down; option i uses
    its first N_i), returns (hold[n, stride + 1, 2] = seller's and buyer's stock holdings after
    rebalancing at t = 0..N_i, NaN beyond and after the buyer stops; cash[n, stride + 1, 2] =
    their cash after rebalancing, in time-t money, of the self-financing portfolios that start
    from the ask and from minus the bid, NaN where hold is; stop[n] = the buyer's stopping time
    or -1; status[n])."""
    a = _as_table(opts)
    n = a.shape[0]
    mv = np.ascontiguousarray(moves, np.int8).reshape(n, -1)
    stride = mv.shape[1]
    hold = np.empty((n, stride + 1, 2), np.float64)
    cash = np.empty((n, stride + 1, 2), np.float64)
    stop = np.empty(n, np.int32)
    st = np.empty(n, np.int32)
    _load().or_hedge_path(_ptr(a), n, _ptr(mv), stride, _ptr(hold), _ptr(cash), _ptr(stop), _ptr(st),
                          _threads(nthreads))
    return hold, cash, stop, st


def root_objective(opt, party: int, ys):
    """F(y) + S0 y at the root (F = w_0/r of the seller, party 0, or the buyer, party 1): the
    value a hedge to holding y attains."""
    a = _as_table(opt)[:1]
    y = np.ascontiguousarray(np.atleast_1d(ys), np.float64)
    out = np.empty_like(y)
    rc = _load().or_root_objective(_ptr(a), int(party), _ptr(y), len(y), _ptr(out))
    if rc:
        raise ValueError("oracle error %d" % rc)
    return out


# ---------------------------------------------------------------- Algorithm 1
def alg1_price(opt, threads: int, L: int, crr: bool = False):
    """One option by the paper's parallel scheme (Section 4.2, Algorithm 1) on `threads`
    threads with blocks of at most L levels, over the same node steps as price_ask_bid
    (crr=False: returns ([ask, bid], status, nodes per thread)) or crr_price (crr=True:
    returns ([price], status, nodes per thread))."""
    a = _as_table(opt)[:1]
    out = np.empty(1 if crr else 2, np.float64)
    st = np.zeros(1, np.int32)
    per = np.zeros(max(int(threads), 1), np.int64)
    f = _load().or_alg1_crr if crr else _load().or_alg1_tc
    f(_ptr(a), int(threads), int(L), _ptr(out), _ptr(st), _ptr(per))
    return out, int(st[0]), per


def alg1_rounds(top: int, threads: int, L: int):
    """The rounds of Algorithm 1 from base level `top`: a list of (B, D, active threads)."""
    cap = 4 * (top + 2)
    buf = np.zeros(3 * cap, np.int32)
    n = _load().or_alg1_rounds(int(top), int(threads), int(L), _ptr(buf), cap)
    return [tuple(int(v) for v in buf[3 * k:3 * k + 3]) for k in range(n)]


# ---------------------------------------------------------------- PL primitives
class PL:
    """A piecewise-linear function: breakpoints y (strictly increasing), values f, tail slopes."""

    def __init__(self, y, f, sL, sR):
        self.y = np.ascontiguousarray(y, np.float64)
        self.f = np.ascontiguousarray(f, np.float64)
        self.sL = float(sL)
        self.sR = float(sR)

    def __call__(self, x):
        x = np.ascontiguousarray(np.atleast_1d(x), np.float64)
        out = np.empty_like(x)
        rc = _load().or_pl_eval(_ptr(self.y), _ptr(self.f), len(self.y), self.sL, self.sR,
                                _ptr(x), len(x), _ptr(out))
        if rc:
            raise ValueError("oracle error %d" % rc)
        return out

    def __repr__(self):
        return "PL(y=%r, f=%r, sL=%r, sR=%r)" % (self.y.tolist(), self.f.tolist(), self.sL, self.sR)


def _result(rc, yo, fo, sL, sR):
    if rc < 0:
        raise ValueError("oracle error %d" % rc)
    return PL(yo[:rc].copy(), fo[:rc].copy(), sL.value, sR.value)


def _bufs(cap):
    return (np.empty(cap, np.float64), np.empty(cap, np.float64), ctypes.c_double(),
            ctypes.c_double())


def envelope(F: PL, G: PL, take_max: bool) -> PL:
    cap = 4 * (len(F.y) + len(G.y)) + 8
    yo, fo, sL, sR = _bufs(cap)
    rc = _load().or_pl_envelope(_ptr(F.y), _ptr(F.f), len(F.y), F.sL, F.sR, _ptr(G.y), _ptr(G.f),
                                len(G.y), G.sL, G.sR, 1 if take_max else 0, _ptr(yo), _ptr(fo),
                                cap, ctypes.byref(sL), ctypes.byref(sR))
    return _result(rc, yo, fo, sL, sR)


def restrict(F: PL, Sa: float, Sb: float) -> PL:
    cap = 8 * len(F.y) + 8
    yo, fo, sL, sR = _bufs(cap)
    rc = _load().or_pl_restrict(_ptr(F.y), _ptr(F.f), len(F.y), F.sL, F.sR, float(Sa), float(Sb),
                                _ptr(yo), _ptr(fo), cap, ctypes.byref(sL), ctypes.byref(sR))
    return _result(rc, yo, fo, sL, sR)


def rebalance(F: PL, Sa, Sb, y0=0.0):
    """The holding y' that attains inf_y' [F(y') + theta(y' - y0)] (theta: buy at Sa, sell at
    Sb; the rightmost among equal minima) and that infimum."""
    yo, vo = ctypes.c_double(), ctypes.c_double()
    rc = _load().or_pl_rebalance(_ptr(F.y), _ptr(F.f), len(F.y), F.sL, F.sR, float(Sa), float(Sb),
                                 float(y0), ctypes.byref(yo), ctypes.byref(vo))
    if rc:
        raise ValueError("oracle error %d" % rc)
    return yo.value, vo.value


def node_step(zu: PL, zd: PL, r, Sa, Sb, xi, zeta, buyer: bool) -> PL:
    cap = 16 * (len(zu.y) + len(zd.y)) + 16
    yo, fo, sL, sR = _bufs(cap)
    rc = _load().or_node_step(_ptr(zu.y), _ptr(zu.f), len(zu.y), zu.sL, zu.sR, _ptr(zd.y),
                              _ptr(zd.f), len(zd.y), zd.sL, zd.sR, float(r), float(Sa), float(Sb),
                              float(xi), float(zeta), 1 if buyer else 0, _ptr(yo), _ptr(fo), cap,
                              ctypes.byref(sL), ctypes.byref(sR))
    return _result(rc, yo, fo, sL, sR)
