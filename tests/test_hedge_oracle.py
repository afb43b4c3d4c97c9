"""Pins of the oracle's hedge at the root (Section 3: the rebalancing a hedger makes, v(y) =
inf over y' of w/r at y' plus the cost of moving from y to y'), against what the paper and
the mathematics fix:

  * the paper's one-step examples (Section 3): the seller with w = max(z^u, z^d) moves to
    y' = -1 and v(0) = 130/1.18 - 80 < u(0) = 50, so immediate exercise sets the ask; the
    buyer moves to y' = +1 and v(0) = 120 - 130/1.18 > u(0) = -10, so the buyer exercises;
  * without costs the functions at t = 1 are lines V - y S, so the hedge is the CRR delta
    (V_u - V_d) / (S0 u - S0 d) for the seller and its negative for the buyer, with V_u, V_d
    from a textbook CRR recursion written here;
  * the rebalancing target on random PL functions against a dense grid search of the
    objective (convex and non-convex, with and without a kink at the starting holding).
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _pl(d):
    return oracle.PL([d["kink"]], [d["value"]], d["sL"], d["sR"])


def test_paper_one_step_examples():
    with open(os.path.join(GOLD, "paper_one_step.json")) as f:
        g = json.load(f)
    r = 1.18  # the example's r: p = 0.9454 = (r - d)/(u - d) with u = 1.2
    # seller: w = max(z^u, z^d) has its kink at y = -1; rebalancing from no stock goes there
    s = g["seller"]
    w = oracle.envelope(_pl(s["zu"]), _pl(s["zd"]), True)
    F = oracle.PL(w.y, w.f / r, w.sL / r, w.sR / r)
    y, v = oracle.rebalance(F, s["Sa"], s["Sb"], 0.0)
    assert y == -1.0
    assert abs(v - (130.0 / r - s["Sb"])) < 1e-12
    assert s["ask"] > v  # u(0) = 50 = ask: set by immediate exercise
    # buyer: the kink at y = +1
    b = g["buyer"]
    w = oracle.envelope(_pl(b["zu"]), _pl(b["zd"]), True)
    F = oracle.PL(w.y, w.f / r, w.sL / r, w.sR / r)
    y, v = oracle.rebalance(F, b["Sa"], b["Sb"], 0.0)
    assert y == 1.0
    assert abs(v - (b["Sa"] - 130.0 / r)) < 1e-12
    assert -b["bid"] < v  # u(0) = -10 = -bid: the buyer exercises


def _crr_level1(o):
    """Textbook American CRR values at t = 1 (no costs), in plain numpy."""
    N = int(o["N"])
    dt = o["T"] / N
    u = np.exp(o["sigma"] * np.sqrt(dt))
    d = 1.0 / u
    r = np.exp(o["R"] * dt)
    p = (r - d) / (u - d)

    def payoff(S):
        if o["payoff"] == W.PUT:
            return o["K"] - S
        if o["payoff"] == W.CALL:
            return S - o["K"]
        return np.maximum(S - o["K"], 0.0) - np.maximum(S - o["K2"], 0.0)

    j = np.arange(N + 1)
    V = np.maximum(payoff(o["S0"] * u ** (2 * j - N)), 0.0)
    for t in range(N - 1, 0, -1):
        j = np.arange(t + 1)
        V = np.maximum(payoff(o["S0"] * u ** (2 * j - t)), (p * V[1:] + (1 - p) * V[:-1]) / r)
    return V[1], V[0], o["S0"] * u, o["S0"] * d, payoff(o["S0"]), (p * V[1] + (1 - p) * V[0]) / r


@pytest.mark.parametrize("payoff", [W.PUT, W.CALL, W.SPREAD])
def test_no_costs_hedge_is_crr_delta(payoff):
    rng = np.random.default_rng(77 + payoff)
    for _ in range(12):
        o = W.make(S0=float(rng.uniform(80, 120)), K=100.0, K2=110.0, sigma=float(rng.uniform(0.1, 0.5)),
                   R=float(rng.uniform(0.0, 0.1)), T=float(rng.uniform(0.1, 2.0)), k=0.0,
                   N=int(rng.integers(2, 160)), payoff=payoff)[0]
        h, st = oracle.initial_hedge(o)
        assert st[0] == 0
        Vu, Vd, Su, Sd, ex, cont = _crr_level1(o)
        delta = (Vu - Vd) / (Su - Sd)
        scale = max(1.0, abs(delta))
        assert abs(h[0, 0] - delta) <= 1e-9 * scale, (h, delta)
        assert abs(h[0, 1] + delta) <= 1e-9 * scale, (h, delta)
        if abs(ex - cont) > 1e-9 * max(1.0, abs(cont)):
            assert h[0, 2] == (1.0 if ex > cont else 0.0)  # immediate exercise sets the price
            assert h[0, 3] == h[0, 2]                       # and the buyer takes it


def test_deep_in_the_money_put_exercises_at_once():
    o = W.make(S0=50.0, K=100.0, k=0.0, N=60, R=0.08)
    h, st = oracle.initial_hedge(o)
    assert st[0] == 0 and h[0, 2] == 1.0 and h[0, 3] == 1.0


def test_rebalance_against_grid_search():
    rng = np.random.default_rng(5)
    for trial in range(200):
        m = int(rng.integers(1, 7))
        y = np.sort(rng.uniform(-3, 3, m))
        if m > 1 and np.min(np.diff(y)) < 1e-3:
            continue
        f = rng.uniform(-5, 5, m)
        Sa = float(rng.uniform(1.0, 3.0))
        Sb = float(rng.uniform(0.2, Sa))
        sL = -Sb - float(rng.uniform(0.1, 2.0))  # tails rise away from the breakpoints
        sR = -Sa + float(rng.uniform(0.1, 2.0))
        y0 = float(rng.choice([0.0, rng.uniform(-3, 3)]))
        F = oracle.PL(y, f, sL, sR)
        ys, vs = oracle.rebalance(F, Sa, Sb, y0)
        grid = np.concatenate([np.linspace(-8, 8, 160001), y, [y0]])
        obj = F(grid) + np.where(grid >= y0, Sa, Sb) * (grid - y0)
        assert vs <= obj.min() + 1e-12, trial
        assert abs(vs - obj.min()) <= 1e-12 * max(1.0, abs(vs)), trial
        at = F(np.array([ys]))[0] + (Sa if ys >= y0 else Sb) * (ys - y0)
        assert abs(at - vs) <= 1e-12 * max(1.0, abs(vs)), trial


def _crr_tree(o):
    """Textbook American CRR values V[t][j] for t <= N (plain numpy), the stock prices, the
    exercise values and the continuation values."""
    N = int(o["N"])
    dt = o["T"] / N
    u = np.exp(o["sigma"] * np.sqrt(dt))
    d = 1.0 / u
    r = np.exp(o["R"] * dt)
    p = (r - d) / (u - d)

    def payoff(S):
        if o["payoff"] == W.PUT:
            return o["K"] - S
        if o["payoff"] == W.CALL:
            return S - o["K"]
        return np.maximum(S - o["K"], 0.0) - np.maximum(S - o["K2"], 0.0)

    S = [o["S0"] * u ** (2 * np.arange(t + 1) - t) for t in range(N + 2)]
    V = [None] * (N + 2)
    cont = [None] * (N + 1)
    V[N + 1] = np.zeros(N + 2)
    V[N] = np.maximum(payoff(S[N]), 0.0)
    cont[N] = np.zeros(N + 1)
    for t in range(N - 1, -1, -1):
        cont[t] = (p * V[t + 1][1:] + (1 - p) * V[t + 1][:-1]) / r
        V[t] = np.maximum(payoff(S[t]), cont[t])
    return S, V, cont, [payoff(S[t]) for t in range(N + 1)]


@pytest.mark.parametrize("payoff", [W.PUT, W.CALL, W.SPREAD])
def test_no_costs_path_hedge_is_crr_delta_and_exercise_boundary(payoff):
    """Without costs the hedge along any path is the CRR delta of the path's node at every
    step (the seller's; the buyer's is its negative), and the buyer stops at the first node of
    the path where exercise beats continuation."""
    rng = np.random.default_rng(91 + payoff)
    for _ in range(8):
        N = int(rng.integers(2, 90))
        o = W.make(S0=float(rng.uniform(70, 130)), K=100.0, K2=110.0, sigma=float(rng.uniform(0.1, 0.5)),
                   R=float(rng.uniform(0.0, 0.1)), T=float(rng.uniform(0.1, 2.0)), k=0.0, N=N,
                   payoff=payoff)
        mv = rng.integers(0, 2, (1, N)).astype(np.int8)
        hold, stop, st = oracle.hedge_path(o, mv)
        assert st[0] == 0
        S, V, cont, ex = _crr_tree(o[0])
        j = 0
        want_stop = -1
        for t in range(N + 1):
            delta = (V[t + 1][j + 1] - V[t + 1][j]) / (S[t + 1][j + 1] - S[t + 1][j])
            scale = max(1.0, abs(delta))
            assert abs(hold[0, t, 0] - delta) <= 1e-9 * scale, (t, hold[0, t], delta)
            gap = ex[t][j] - cont[t][j]
            if want_stop < 0:
                if abs(gap) <= 1e-9 * max(1.0, abs(cont[t][j])):
                    break  # a tie between exercise and continuation: either choice is optimal
                if gap > 0:
                    want_stop = t
                else:
                    assert abs(hold[0, t, 1] + delta) <= 1e-9 * scale, (t, hold[0, t], delta)
            if t < N:
                j += int(mv[0, t])
        else:
            assert stop[0] == want_stop, (stop[0], want_stop)


def test_path_hedge_starts_with_the_root_hedge():
    t = W.random_table(20, 6060, N_lo=2, N_hi=120)
    mv = np.random.default_rng(3).integers(0, 2, (len(t), int(t["N"].max()))).astype(np.int8)
    hold, stop, st = oracle.hedge_path(t, mv, nthreads=4)
    h0, st0 = oracle.initial_hedge(t, nthreads=4)
    assert np.array_equal(st, st0)
    ok = st == 0
    assert np.array_equal(hold[ok, 0, 0], h0[ok, 0])
    buyer_at_root = np.where(stop[ok] == 0, np.nan, h0[ok, 1])
    assert np.array_equal(hold[ok, 0, 1], buyer_at_root, equal_nan=True)
    assert np.all((stop[ok] == 0) == (h0[ok, 3] == 1.0))
