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
    objective (convex and non-convex, with and without a kink at the starting holding);
  * along a path, the defining property of the two prices (Section 3): the seller's
    self-financing portfolio started from the ask with the path's holdings can settle an
    exercise at every node and its stock at N+1, and the buyer's, started from minus the
    bid, can settle the buyer's exercise at its stopping node (or its stock at N+1); the
    settlement costs are written out here from the payoff and the bid/ask prices.
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
        hold, cash, stop, st = oracle.hedge_path(o, mv)
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
    hold, cash, stop, st = oracle.hedge_path(t, mv, nthreads=4)
    h0, st0 = oracle.initial_hedge(t, nthreads=4)
    assert np.array_equal(st, st0)
    ok = st == 0
    assert np.array_equal(hold[ok, 0, 0], h0[ok, 0])
    buyer_at_root = np.where(stop[ok] == 0, np.nan, h0[ok, 1])
    assert np.array_equal(hold[ok, 0, 1], buyer_at_root, equal_nan=True)
    assert np.all((stop[ok] == 0) == (h0[ok, 3] == 1.0))


def _settle(o, S, kt, x, y, buyer):
    """Cash left after settling the payoff at a node with stock price S and cost rate kt,
    from cash x and y shares, then closing the stock position: the seller pays (xi, zeta),
    the buyer receives it (Eq. 1, Eq. 6).  Shares are bought at (1+kt) S, sold at (1-kt) S."""
    if o["payoff"] == W.PUT:
        xi, zeta = o["K"], -1.0
    elif o["payoff"] == W.CALL:
        xi, zeta = -o["K"], 1.0
    else:
        xi, zeta = max(S - o["K"], 0.0) - max(S - o["K2"], 0.0), 0.0
    if buyer:
        x, q = x + xi, y + zeta
    else:
        x, q = x - xi, y - zeta
    return x + q * (1.0 - kt) * S if q >= 0 else x + q * (1.0 + kt) * S


def _no_payoff(o):
    a = dict(zip(o.dtype.names, o.tolist()))
    a["payoff"], a["K"], a["K2"] = W.SPREAD, 1e300, 1e300  # xi = 0, zeta = 0
    return a


@pytest.mark.parametrize("payoff", [W.PUT, W.CALL, W.SPREAD])
def test_path_portfolios_superhedge(payoff):
    rng = np.random.default_rng(404 + payoff)
    t = W.random_table(16, 505 + payoff, N_lo=2, N_hi=160, payoffs=(payoff,), k_hi=0.03)
    mv = rng.integers(0, 2, (len(t), int(t["N"].max()))).astype(np.int8)
    hold, cash, stop, st = oracle.hedge_path(t, mv, nthreads=4)
    ask_bid, pst = oracle.price_ask_bid(t, nthreads=4)
    assert np.all(st == 0) and np.all(pst == 0)
    for i, o in enumerate(t):
        N = int(o["N"])
        dt = o["T"] / N
        u = np.exp(o["sigma"] * np.sqrt(dt))
        r = np.exp(o["R"] * dt)
        ask, bid = ask_bid[i]
        jt = np.concatenate([[0], np.cumsum(mv[i, :N] != 0)])

        def S(tt, j):
            return o["S0"] * u ** (2 * j - tt)

        def tol(x, y, s):
            return 1e-9 * max(1.0, abs(x), s * abs(y))

        # the seller: cash before the rebalancing at t is r x_{t-1} (the ask at t = 0)
        x, y = ask, 0.0
        for tt in range(N + 1):
            kt = 0.0 if tt == 0 else o["k"]
            s = S(tt, jt[tt])
            left = _settle(o, s, kt, x, y, False)
            assert left >= -tol(x, y, s), (i, tt, x, y, left)
            x, y = cash[i, tt, 0] * r, hold[i, tt, 0]
        for j in (jt[N], jt[N] + 1):  # both nodes of the extra instant N+1
            s = S(N + 1, j)
            left = _settle(_no_payoff(o), s, o["k"], x, y, False)
            assert left >= -tol(x, y, s), (i, "N+1", x, y, left)
        # the buyer: cash before the rebalancing at t is r x_{t-1} (minus the bid at t = 0)
        x, y = -bid, 0.0
        tau = int(stop[i])
        assert tau == -1 or np.all(np.isnan(hold[i, tau:N + 1, 1]))
        last = N if tau < 0 else tau - 1
        assert not np.any(np.isnan(hold[i, :last + 1, 1]))
        for tt in range(last + 1):
            x, y = cash[i, tt, 1] * r, hold[i, tt, 1]
        if tau >= 0:
            s = S(tau, jt[tau])
            if tau == 0:
                x, y = -bid, 0.0
            left = _settle(o, s, 0.0 if tau == 0 else o["k"], x, y, True)
            assert left >= -tol(x, y, s), (i, "stop", tau, x, y, left)
        else:
            for j in (jt[N], jt[N] + 1):
                s = S(N + 1, j)
                left = _settle(_no_payoff(o), s, o["k"], x, y, True)
                assert left >= -tol(x, y, s), (i, "N+1 buyer", x, y, left)



def _node_functions(o, buyer):
    """z_t at every node of a small tree, built level by level with the oracle's node step
    (itself pinned by the price tests): z[t][j], t = 0..N+1."""
    N = int(o["N"])
    dt = o["T"] / N
    u = np.exp(o["sigma"] * np.sqrt(dt))
    r = np.exp(o["R"] * dt)
    z = [None] * (N + 2)
    z[N + 1] = []
    for j in range(N + 2):
        S = o["S0"] * u ** (2 * j - N - 1)
        z[N + 1].append(oracle.PL([0.0], [0.0], -(1 + o["k"]) * S, -(1 - o["k"]) * S))
    for t in range(N, -1, -1):
        kt = 0.0 if t == 0 else o["k"]
        z[t] = []
        for j in range(t + 1):
            S = o["S0"] * u ** (2 * j - t)
            if o["payoff"] == W.PUT:
                xi, zeta = o["K"], -1.0
            elif o["payoff"] == W.CALL:
                xi, zeta = -o["K"], 1.0
            else:
                xi, zeta = max(S - o["K"], 0.0) - max(S - o["K2"], 0.0), 0.0
            z[t].append(oracle.node_step(z[t + 1][j + 1], z[t + 1][j], r, (1 + kt) * S, (1 - kt) * S,
                                         xi, zeta, buyer))
    return z, u, r


@pytest.mark.parametrize("party", [0, 1])
def test_path_portfolios_are_tight_on_the_binding_path(party):
    """The portfolios start from exactly the price, so they carry no slack where the price is
    attained: following at each level the successor whose z is larger at the holding (the one
    that sets w = max(z_up, z_down)), the cash before rebalancing equals z_t at the holding
    the party arrives with, until exercise binds (z_t = u_t there).  Catches cash that is too
    high (a rebalancing charged too little) as the superhedging pins catch cash too low."""
    t = W.concat(W.make(N=10, k=0.01, payoff=W.PUT, S0=95.0), W.make(N=12, k=0.02, payoff=W.CALL),
                 W.make(N=9, k=0.005, payoff=W.SPREAD, K=95.0, K2=105.0, sigma=0.3),
                 W.make(N=11, k=0.015, payoff=W.PUT, S0=110.0, R=0.02),
                 W.make(N=8, k=0.03, payoff=W.CALL, S0=90.0, sigma=0.4))
    checked = 0
    for i, o in enumerate(t):
        N = int(o["N"])
        z, u, r = _node_functions(o, party == 1)
        moves = np.zeros((1, N), np.int8)
        for tt in range(N):  # the binding successor at each level, given the holding there
            hold, cash, stop, st = oracle.hedge_path(t[i:i + 1], moves)
            y = hold[0, tt, party]
            if np.isnan(y):
                break
            j = int(moves[0, :tt].sum())
            moves[0, tt] = 1 if z[tt + 1][j + 1](y)[0] >= z[tt + 1][j](y)[0] else 0
        hold, cash, stop, st = oracle.hedge_path(t[i:i + 1], moves)
        ask_bid, _ = oracle.price_ask_bid(t[i:i + 1])
        C = ask_bid[0, 0] if party == 0 else -ask_bid[0, 1]
        y, j = 0.0, 0
        for tt in range(N + 2):
            if tt == N + 1:  # the extra instant: the binding node of the two
                j = j + 1 if z[N + 1][j + 1](y)[0] >= z[N + 1][j](y)[0] else j
            elif tt > 0:
                j += int(moves[0, tt - 1])
            S = o["S0"] * u ** (2 * j - tt)
            zt = z[tt][j](y)[0]
            scale = max(1.0, abs(C), S * abs(y))
            assert abs(C - zt) <= 1e-9 * scale, (i, party, tt, C, zt)
            checked += 1
            kt = 0.0 if tt == 0 else o["k"]
            oo = o if tt <= N else _no_payoff(o)
            if abs(zt + _settle(oo, S, kt, 0.0, y, party == 1)) <= 1e-9 * scale:
                break  # exercise (or the final settlement) binds here
            if tt == N + 1 or np.isnan(hold[0, tt, party]):
                break
            C, y = cash[0, tt, party] * r, hold[0, tt, party]
    assert checked >= 2 * len(t)


EXACT_PATH_CASES = [
    dict(k=0.01, N=8, payoff=W.PUT),
    dict(k=0.03, N=7, payoff=W.PUT, S0=92.0, R=0.08),
    dict(k=0.01, N=9, payoff=W.CALL),
    dict(k=0.02, N=6, payoff=W.CALL, S0=108.0, sigma=0.35),
    dict(K=95.0, K2=105.0, k=0.01, N=8, payoff=W.SPREAD),
    dict(K=95.0, K2=105.0, k=0.02, N=7, payoff=W.SPREAD, sigma=0.1, T=0.1),
]


@pytest.mark.parametrize("case", EXACT_PATH_CASES)
def test_path_hedge_matches_exact_arithmetic(case):
    """The oracle's hedge along a path against exact rational arithmetic (oracle/exact.py: the
    induction with an exact slope restriction written from its definition, and the
    rebalancing by exact comparison of the candidates, the rightmost among exact ties), on 6
    paths per option with costs: holdings within 1e-9 of max(1, |y|), cash within 1e-9 of
    max(|x|, S0), NaN exactly where the buyer has stopped, the same stopping level."""
    from oracle import exact
    t = W.make(**case)
    o = t[0]
    N = int(o["N"])
    rng = np.random.default_rng(int(1000 * case["k"]) + N)
    paths = [np.ones(N, np.int8), np.zeros(N, np.int8)] + [rng.integers(0, 2, N).astype(np.int8)
                                                           for _ in range(4)]
    for mv in paths:
        hold, cash, stop, st = oracle.hedge_path(t, mv[None, :])
        assert st[0] == 0
        a, b, eh, ec, es = exact.hedge_path(o, mv)
        assert stop[0] == es, (stop[0], es)
        for tt in range(N + 1):
            for p in (0, 1):
                ye, xe = eh[tt][p], ec[tt][p]
                y, x = hold[0, tt, p], cash[0, tt, p]
                if ye is None:
                    assert np.isnan(y) and np.isnan(x), (tt, p)
                    continue
                assert abs(y - float(ye)) <= 1e-9 * max(1.0, abs(float(ye))), (tt, p, y, float(ye))
                assert abs(x - float(xe)) <= 1e-9 * max(abs(float(xe)), float(o["S0"])), (tt, p, x, float(xe))
