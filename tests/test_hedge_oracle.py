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
