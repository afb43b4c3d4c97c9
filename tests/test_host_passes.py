"""The kernel's level passes compiled for the host with a one-lane team (tests/host_passes.cpp)
against the oracle: prices at the parity tolerance, the same points whether a level is split
over 1 or G teams (bitwise), the adjoint against the oracle's dual-number gradient, and the
hedge along a path against the oracle's.  This checks the passes' logic (merge with owner
handoff, running minima, restriction and exercise per piece, the split of a level, the
reverse sweep, the path's w kept per level and the forward rebalancing) without a GPU."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RTOL = 1e-10
_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        out = os.path.join(tempfile.mkdtemp(prefix="hostpasses"), "libhostpasses.so")
        src = os.path.join(ROOT, "tests", "host_passes.cpp")
        inc = os.path.join(ROOT, "paper_1110_2477_gb300", "csrc")
        r = subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", inc, "-o", out, src],
                           capture_output=True, text=True)
        if r.returncode != 0:
            pytest.fail("g++ failed: " + r.stderr[-2000:])
        _LIB = ctypes.CDLL(out)
    return _LIB


def _rec(row):
    return np.ascontiguousarray(np.array([row], dtype=W.OPTION_DTYPE))


def _price(row, G=0):
    a = _rec(row)
    out = np.zeros(2)
    pts = np.zeros(3, np.int64)
    P = ctypes.c_void_p
    if G:
        rc = _lib().hp_price_split(a.ctypes.data_as(P), G, out.ctypes.data_as(P), pts.ctypes.data_as(P))
    else:
        rc = _lib().hp_price(a.ctypes.data_as(P), out.ctypes.data_as(P), pts.ctypes.data_as(P))
    return rc, out, pts


def _table():
    return W.concat(W.random_table(24, 31000, N_lo=1, N_hi=90, k_hi=0.05),
                    W.make(S0=100, K=95, K2=105, sigma=0.1, T=0.1, k=0.02, N=60, payoff=W.SPREAD),
                    W.make(S0=100, K=100, sigma=0.1, T=0.1, k=0.02, N=60, payoff=W.CALL),
                    W.make(k=0.0, N=40), W.make(k=0.01, N=1), W.make(R=5.0, N=2, T=1.0))


def test_host_passes_match_oracle():
    t = _table()
    ref, rst = oracle.price_ask_bid(t, nthreads=4)
    for i in range(len(t)):
        rc, out, _ = _price(t[i])
        assert rc == rst[i], (i, rc, rst[i])
        if rc == 0:
            scale = np.maximum(np.abs(ref[i]), 1e-2 * t["K"][i])
            assert np.all(np.abs(out - ref[i]) <= RTOL * scale), (i, out, ref[i])


@pytest.mark.parametrize("G", [2, 3, 16])
def test_level_split_over_teams_is_bitwise_equal(G):
    t = _table()
    for i in range(len(t)):
        rc1, out1, pts1 = _price(t[i])
        rc2, out2, pts2 = _price(t[i], G)
        assert rc1 == rc2
        if rc1 == 0:
            assert np.array_equal(out1.view(np.int64), out2.view(np.int64))
            assert np.array_equal(pts1, pts2)


@pytest.mark.parametrize("cap", [3, 8, 40, 600])
def test_fused_level_step_is_bitwise_equal(cap):
    """Passes 1-3 per chunk of whole nodes with w in a small on-chip array (chunks of a few
    nodes, nodes too large for the array on the global path, chunks whose w outgrows the
    array rerun globally) give the same bits and point counts as the one-pass level."""
    t = _table()
    P = ctypes.c_void_p
    for i in range(len(t)):
        rc1, out1, pts1 = _price(t[i])
        a = _rec(t[i])
        out2 = np.zeros(2)
        pts2 = np.zeros(3, np.int64)
        rc2 = _lib().hp_price_chip(a.ctypes.data_as(P), cap, out2.ctypes.data_as(P), pts2.ctypes.data_as(P))
        assert rc1 == rc2
        if rc1 == 0:
            assert np.array_equal(out1.view(np.int64), out2.view(np.int64)), (i, out1, out2)
            assert np.array_equal(pts1, pts2)


@pytest.mark.parametrize("G,Dmax,light,colp", [(1, 8, 1 << 30, 1 << 30), (2, 3, 1 << 30, 1 << 30),
                                                (3, 8, 1 << 30, 1 << 30), (7, 2, 1 << 30, 1 << 30),
                                                (16, 8, 1 << 30, 1 << 30), (5, 8, 6, 1 << 30),
                                                (4, 1, 1 << 30, 1 << 30), (3, 8, 0, 1 << 30),
                                                (9, 8, 1 << 30, 5)])
def test_trapezoid_rounds_are_bitwise_equal(G, Dmax, light, colp):
    """The whole-GPU form's trapezoid rounds (TcTrap: each team copies a window of columns of
    the complete level, split by points, and goes down up to Dmax levels on it, recomputing
    the halo columns its right neighbour owns), alone or mixed with single levels (light: the
    points a team, colp: the points a column, below which a level is taken in a round),
    give the bits of the single-team run."""
    t = _table()
    P = ctypes.c_void_p
    for i in range(len(t)):
        rc1, out1, _ = _price(t[i])
        a = _rec(t[i])
        out2 = np.zeros(2)
        pts = np.zeros(3, np.int64)
        rounds = np.zeros(2, np.int32)
        rc2 = _lib().hp_price_trap(a.ctypes.data_as(P), G, Dmax, light, colp, out2.ctypes.data_as(P),
                                   pts.ctypes.data_as(P), rounds.ctypes.data_as(P))
        assert rc1 == rc2, (i, rc1, rc2)
        if rc1 == 0:
            assert np.array_equal(out1.view(np.int64), out2.view(np.int64)), (i, out1, out2)
            if light >= (1 << 30) and colp >= (1 << 30):
                assert rounds[1] == 0 and rounds[0] >= (t["N"][i] + 1) // Dmax
            if light == 0:
                assert rounds[0] == 0


@pytest.mark.parametrize("G", [1, 2, 3, 5, 16, 61])
def test_nodes_split_over_teams_are_bitwise_equal(G):
    """Every level with its nodes split over G teams at the quantiles of the merged successor
    points (TcSplit: shares that begin and end inside nodes, the owner carry recomputed, the
    running minima combined across shares, the neighbouring shares' boundary points for the
    pieces that cross a boundary), with as many teams as points at the top of the tree (empty
    shares), give the bits and the point counts of the single-team run."""
    t = W.concat(_table(), W.make(K=95.0, K2=105.0, k=0.03, N=120, sigma=0.1, payoff=W.SPREAD),
                 W.make(k=0.04, N=110, sigma=0.1, payoff=W.CALL))
    P = ctypes.c_void_p
    for i in range(len(t)):
        rc1, out1, pts1 = _price(t[i])
        a = _rec(t[i])
        out2 = np.zeros(2)
        pts2 = np.zeros(3, np.int64)
        rc2 = _lib().hp_price_nsplit(a.ctypes.data_as(P), G, out2.ctypes.data_as(P), pts2.ctypes.data_as(P))
        assert rc1 == rc2, (i, rc1, rc2)
        if rc1 == 0:
            assert np.array_equal(out1.view(np.int64), out2.view(np.int64)), (i, out1, out2)
            assert np.array_equal(pts1, pts2), (i, pts1, pts2)


@pytest.mark.parametrize("payoff", [W.PUT, W.CALL, W.SPREAD])
def test_host_adjoint_matches_oracle_gradient(payoff):
    """The adjoint (line adjoints per piece) against the oracle's gradient on 40 options of
    one payoff, N in [2, 160]: exercise branches in the left tails, running minima at the
    ends of their range, and the crossings of nearly parallel pieces of calls and spreads.
    Both modes: records of every level kept by the forward pass (full), and checkpoints
    with a recomputed segment each; they give the same bits."""
    t = W.random_table(40, 31500 + payoff, N_lo=2, N_hi=160, payoffs=(payoff,))
    t["k"] = np.maximum(t["k"], 1e-4)
    rout, rgrad, rst = oracle.greeks(t, nthreads=8)
    P = ctypes.c_void_p
    for i in range(len(t)):
        a = _rec(t[i])
        res = []
        for full in (1, 0):
            out = np.zeros(2)
            grad = np.zeros(12)
            rc = _lib().hp_greeks(a.ctypes.data_as(P), out.ctypes.data_as(P), grad.ctypes.data_as(P),
                                  full)
            assert rc == rst[i] == 0
            scale = np.maximum(np.abs(rgrad[i].reshape(-1)), 1e-3 * t["K"][i])
            assert np.all(np.abs(grad - rgrad[i].reshape(-1)) <= 1e-6 * scale), (i, full, grad, rgrad[i])
            res.append(np.concatenate([out, grad]))
        assert np.array_equal(res[0].view(np.int64), res[1].view(np.int64)), i


def test_host_hedge_path_matches_oracle():
    """path_one on the host (one-lane team) against the oracle's hedge along a path: prices
    bitwise those of the host pricing run, holdings within 1e-9 of max(1, |y|), cash within
    1e-9 of max(|x|, S0), the same stopping levels; a slice too small for the path store
    gives ST_CAPACITY."""
    t = W.concat(W.random_table(30, 32000, N_lo=1, N_hi=120, k_hi=0.03),
                 W.make(S0=100, K=95, K2=105, sigma=0.1, T=0.1, k=0.02, N=60, payoff=W.SPREAD),
                 W.make(k=0.0, N=40), W.make(k=0.01, N=1))
    S = int(t["N"].max())
    mv = np.random.default_rng(6).integers(0, 2, (len(t), S)).astype(np.int8)
    oh, oc, ostop, ost = oracle.hedge_path(t, mv, nthreads=8)
    P = ctypes.c_void_p
    stops = 0
    for i in range(len(t)):
        N = int(t["N"][i])
        a = _rec(t[i])
        m = np.ascontiguousarray(mv[i])
        out = np.zeros(2)
        hold = np.full(2 * (N + 1), np.nan)
        cash = np.full(2 * (N + 1), np.nan)
        stop = ctypes.c_int(-2)
        rc = _lib().hp_hedge_path(a.ctypes.data_as(P), m.ctypes.data_as(P), 64 << 10, out.ctypes.data_as(P),
                                  hold.ctypes.data_as(P), cash.ctypes.data_as(P), ctypes.byref(stop))
        assert rc == ost[i] == 0, (i, rc)
        prc, pout, _ = _price(t[i])
        assert prc == 0 and np.array_equal(out.view(np.int64), pout.view(np.int64)), i
        assert stop.value == ostop[i], (i, stop.value, ostop[i])
        stops += stop.value >= 0
        h, c = hold.reshape(N + 1, 2), cash.reshape(N + 1, 2)
        ho, co = oh[i, :N + 1], oc[i, :N + 1]
        assert np.array_equal(np.isnan(h), np.isnan(ho)) and np.array_equal(np.isnan(c), np.isnan(co)), i
        f = ~np.isnan(ho)
        assert np.all(np.abs(h[f] - ho[f]) <= 1e-9 * np.maximum(1.0, np.abs(ho[f]))), i
        assert np.all(np.abs(c[f] - co[f]) <= 1e-9 * np.maximum(np.abs(co[f]), t["S0"][i])), i
    assert stops >= 1
    # 64 KiB: too small for the N = 60 spread's level arrays and path store together
    i = len(t) - 3
    out = np.zeros(2)
    hold = np.zeros(2 * 61)
    stop = ctypes.c_int(-2)
    rc = _lib().hp_hedge_path(_rec(t[i]).ctypes.data_as(P), np.ascontiguousarray(mv[i]).ctypes.data_as(P), 64,
                              out.ctypes.data_as(P), hold.ctypes.data_as(P), None, ctypes.byref(stop))
    assert rc == -3


def test_host_root_hedge_matches_oracle():
    """TcRun::root_hedge on the host (one-lane team) against the oracle's hedge at the root:
    holdings within 1e-9 of max(1, |y|), or a breakpoint that attains the same minimum to
    within 1e-12 where two tie; the exercise flags equal wherever u_0(0) and v_0(0) are not
    within rounding of each other (the oracle's root objective decides)."""
    t = W.concat(W.random_table(40, 33000, N_lo=1, N_hi=120, k_hi=0.03), W.make(S0=50.0, N=30, k=0.0),
                 W.make(S0=100, K=95, K2=105, sigma=0.1, T=0.1, k=0.02, N=60, payoff=W.SPREAD))
    oh, ost = oracle.initial_hedge(t, nthreads=8)
    P = ctypes.c_void_p
    for i in range(len(t)):
        out = np.zeros(2)
        hg = np.zeros(4)
        rc = _lib().hp_price_hedge(_rec(t[i]).ctypes.data_as(P), out.ctypes.data_as(P), hg.ctypes.data_as(P))
        assert rc == ost[i] == 0, (i, rc)
        for p in (0, 1):
            yg, yo = hg[p], oh[i, p]
            if abs(yg - yo) > 1e-9 * max(1.0, abs(yo)):
                f = oracle.root_objective(t[i:i + 1], p, [yg, yo])
                assert abs(f[0] - f[1]) <= 1e-12 * max(1.0, abs(f[1])), (i, p, yg, yo, f)
        assert hg[2] in (0.0, 1.0) and hg[3] in (0.0, 1.0)
        # a flag may differ only where exercise and the hedge tie: then the price (ask =
        # max(u, v) for the seller, -bid = min(u, v) for the buyer) equals v to rounding
        if hg[2] != oh[i, 2]:
            v = oracle.root_objective(t[i:i + 1], 0, [oh[i, 0]])[0]
            assert abs(out[0] - v) <= 1e-11 * max(1.0, abs(v)), (i, "seller flag off a tie")
        if hg[3] != oh[i, 3]:
            v = oracle.root_objective(t[i:i + 1], 1, [oh[i, 1]])[0]
            assert abs(-out[1] - v) <= 1e-11 * max(1.0, abs(v)), (i, "buyer flag off a tie")
