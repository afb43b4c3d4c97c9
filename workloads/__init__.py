"""Seeded synthetic option tables.

This module only lays out parameter records and draws them from seeded
generators; it holds none of the pricing arithmetic.  Both the CPU oracle
(tests, CPU baseline) and the GPU library (tests, benchmark) read the tables
it makes.

The paper measures on parameter sets, not on a dataset: the American put and
the cash-settled bull spread of its correctness and performance tests
(Section 5: T=0.25, sigma=0.2, R=0.1, S0=100, K=100 or 95/105), and the
cost-free put of the Appendix (K=100, S0=100, T=3, sigma=0.3, R=0.06).  The
batched tables below widen those into uneven batches.

Record layout (64 bytes, little-endian, matches ``ob_option_t``):
  S0, K, K2, sigma, R, T, k : float64
  N, payoff                 : int32   (payoff 0 = put, 1 = call, 2 = bull spread)
"""
from __future__ import annotations

import numpy as np

OPTION_DTYPE = np.dtype([("S0", "<f8"), ("K", "<f8"), ("K2", "<f8"), ("sigma", "<f8"),
                         ("R", "<f8"), ("T", "<f8"), ("k", "<f8"), ("N", "<i4"),
                         ("payoff", "<i4")])
assert OPTION_DTYPE.itemsize == 64

PUT, CALL, SPREAD = 0, 1, 2
SPREAD_WIDTH = 10.0


def make(S0=100.0, K=100.0, K2=None, sigma=0.2, R=0.1, T=0.25, k=0.005, N=250, payoff=PUT):
    """A one-record table."""
    a = np.zeros(1, OPTION_DTYPE)
    a["S0"], a["K"], a["sigma"], a["R"], a["T"], a["k"] = S0, K, sigma, R, T, k
    a["K2"] = (K + SPREAD_WIDTH) if K2 is None else K2
    a["N"], a["payoff"] = N, payoff
    return a


def concat(*tables):
    return np.concatenate([np.asarray(t, OPTION_DTYPE).reshape(-1) for t in tables])


def single_put_n250():
    """American put with costs, N=250 (the paper's put example), then the same option at k=0."""
    return concat(make(k=0.005, N=250), make(k=0.0, N=250))


def paper_scale(Ns=(1500, 3000, 6000), ks=(0.0025, 0.005, 0.01)):
    """American put (K=100) and cash-settled bull spread (95/105) at paper scale: 2*|ks|*|Ns| rows."""
    rows = []
    for N in Ns:
        for k in ks:
            rows.append(make(K=100.0, k=k, N=N, payoff=PUT))
            rows.append(make(K=95.0, K2=105.0, k=k, N=N, payoff=SPREAD))
    return concat(*rows)


def price_curves(S0s=None, ks=(0.0, 0.0025, 0.005), N=1500):
    """Price curves of the put K=100 (sigma=0.2, R=0.1, T=0.25) over S0 in [90, 110]:
    one row per (S0, k), k varying fastest."""
    if S0s is None:
        S0s = np.linspace(90.0, 110.0, 41)
    return concat(*[make(S0=float(S0), K=100.0, k=float(k), N=N, payoff=PUT) for S0 in S0s for k in ks])


def random_table(n, seed, N_lo=100, N_hi=2000, payoffs=(PUT, CALL, SPREAD), k_hi=0.02,
                 fixed_N=None, k_zero=False):
    """n options with N ~ U{N_lo..N_hi}, S0, K ~ U[80,120], sigma ~ U[0.1,0.5],
    R ~ U[0,0.1], T ~ U[0.1,2], k ~ U[0,k_hi], payoff uniform over ``payoffs``."""
    rng = np.random.default_rng(seed)
    a = np.zeros(n, OPTION_DTYPE)
    a["N"] = rng.integers(N_lo, N_hi + 1, size=n) if fixed_N is None else fixed_N
    a["S0"] = rng.uniform(80.0, 120.0, n)
    a["K"] = rng.uniform(80.0, 120.0, n)
    a["K2"] = a["K"] + SPREAD_WIDTH
    a["sigma"] = rng.uniform(0.1, 0.5, n)
    a["R"] = rng.uniform(0.0, 0.1, n)
    a["T"] = rng.uniform(0.1, 2.0, n)
    a["k"] = 0.0 if k_zero else rng.uniform(0.0, k_hi, n)
    a["payoff"] = rng.choice(np.asarray(payoffs, np.int32), size=n)
    return a


def batched_uneven(n=4096, seed=3):
    """Batched uneven workload: 4096 options, N ~ U{100..2000}, mixed payoffs."""
    return random_table(n, seed)


def greeks_puts(n=1024, seed=4, N=1000):
    """Greeks workload: 1024 American puts, N=1000, batched-table distributions."""
    return random_table(n, seed, payoffs=(PUT,), fixed_N=N)


def crr_puts(n=65536, seed=5, N=2048):
    """Zero-cost limit at scale: 65536 American puts, N=2048, k=0."""
    return random_table(n, seed, payoffs=(PUT,), fixed_N=N, k_zero=True)


def appendix_put(N=20000):
    """The Appendix's cost-free American put: K=100, S0=100, T=3, sigma=0.3, R=0.06."""
    return make(S0=100.0, K=100.0, sigma=0.3, R=0.06, T=3.0, k=0.0, N=N, payoff=PUT)


def node_updates(table, tc=True):
    """Node updates per option: (N+1)(N+2)/2 for the induction with costs (levels 0..N),
    N(N+1)/2 for the plain CRR recursion (levels 0..N-1)."""
    N = np.asarray(table["N"], np.int64)
    return (N + 1) * (N + 2) // 2 if tc else N * (N + 1) // 2
