"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own formulas: the paper's
printed one-step examples, the k = 0 reduction to the textbook CRR price, the
closed-form European binomial sum, the Appendix's printed price, price
orderings and bounds, the exact-rational restatement, brute-force hedging
linear programs on the non-recombining tree, pointwise definitions of the
piecewise-linear primitives, and central differences for the derivatives.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.stats import binom

import oracle
import workloads as W
from oracle import PL, exact, hedging_lp

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _cone(d):
    return PL([d["kink"]], [d["value"]], d["sL"], d["sR"])


# ---------------------------------------------------------------- Section 3 worked examples
def test_one_step_crr_example():
    """Section 3: S_t = 100, u = 1.2, K = 130, p = 0.9454 -> pi_t = max(30, 10.17) = 30.
    A one-step tree with u = exp(sigma sqrt(T/N)) = 1.2 and r = exp(R T/N) = 1.18 (the r
    implied by the printed p) reproduces it."""
    g = _gold("paper_one_step.json")["no_costs"]
    t = W.make(S0=100.0, K=130.0, sigma=math.log(1.2), R=math.log(1.18), T=1.0, k=0.0, N=1)
    am, _ = oracle.crr_price(t, american=True)
    eu, _ = oracle.crr_price(t, american=False)
    u, d, r = 1.2, 1 / 1.2, 1.18
    assert abs((r - d) / (u - d) - g["p_printed"]) < 1e-4  # printed to 4 places
    assert am[0] == pytest.approx(g["price"], abs=1e-12)
    assert round(eu[0], 2) == g["continuation"]


@pytest.mark.parametrize("party", ["seller", "buyer"])
def test_one_step_tc_example(party):
    """Section 3, Eq. 2-8: the seller's and buyer's one-node examples; z_t equals u_t, so
    ask = 50 and bid = 10; pieces -120y+10 / -80y+50 (seller), -120y-10 / -80y-50 (buyer)."""
    g = _gold("paper_one_step.json")[party]
    r = 1.18
    z = oracle.node_step(_cone(g["zu"]), _cone(g["zd"]), r, g["Sa"], g["Sb"], g["xi"], g["zeta"],
                         buyer=(party == "buyer"))
    kink = g["zu"]["kink"]
    (sl, bl), (sr, br) = g["z_pieces"]
    xs = np.array([kink - 3.0, kink - 1.0, kink - 0.25, kink, kink + 0.5, kink + 2.0])
    want = np.where(xs < kink, bl + sl * xs, br + sr * xs)
    np.testing.assert_allclose(z(xs), want, rtol=0, atol=1e-12)
    assert z.sL == sl and z.sR == sr
    if party == "seller":
        assert z(0.0)[0] == pytest.approx(g["ask"], abs=1e-12)
    else:
        assert -z(0.0)[0] == pytest.approx(g["bid"], abs=1e-12)


def test_one_step_restriction_seller():
    """The discounted successor max of the seller example has its kink at y = -1 with value
    130/r and slopes -144/r, -66.67/r; restricting slopes to [-120, -80] gives
    v = 130/r + 120(y+1)^- - 80(y+1)^+ (slopes clipped, kink kept)."""
    g = _gold("paper_one_step.json")["seller"]
    r = 1.18
    w = oracle.envelope(_cone(g["zu"]), _cone(g["zd"]), take_max=True)
    assert w.sL == -144.0 and w.sR == g["zd"]["sR"]
    f = PL(w.y, w.f / r, w.sL / r, w.sR / r)
    v = oracle.restrict(f, 120.0, 80.0)
    xs = np.linspace(-4, 3, 29)
    want = 130.0 / r + np.where(xs < -1, -120.0 * (xs + 1), -80.0 * (xs + 1))
    np.testing.assert_allclose(v(xs), want, rtol=0, atol=1e-11)


# ---------------------------------------------------------------- PL primitives vs definitions
def _random_pl(rng, m, convex=False, slope_lo=-150.0, slope_hi=-50.0):
    y = np.sort(rng.uniform(-3, 3, m))
    while np.any(np.diff(y) <= 1e-6):
        y = np.sort(rng.uniform(-3, 3, m))
    s = rng.uniform(slope_lo, slope_hi, m + 1)
    if convex:
        s = np.sort(s)
    f = np.empty(m)
    f[0] = rng.uniform(0, 50)
    for i in range(1, m):
        f[i] = f[i - 1] + s[i] * (y[i] - y[i - 1])
    return PL(y, f, s[0], s[-1])


def _grid(*fs):
    pts = np.concatenate([f.y for f in fs])
    extra = np.linspace(pts.min() - 2, pts.max() + 2, 301)
    return np.unique(np.concatenate([pts, extra, pts + 1e-4, pts - 1e-4]))


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("take_max", [True, False])
def test_envelope_is_pointwise(seed, take_max):
    rng = np.random.default_rng(seed)
    F = _random_pl(rng, int(rng.integers(1, 9)))
    G = _random_pl(rng, int(rng.integers(1, 9)))
    E = oracle.envelope(F, G, take_max)
    xs = _grid(F, G, E)
    want = np.maximum(F(xs), G(xs)) if take_max else np.minimum(F(xs), G(xs))
    np.testing.assert_allclose(E(xs), want, rtol=0, atol=1e-9)
    assert np.all(np.diff(E.y) > 0)


def _restrict_bruteforce(F, Sa, Sb, xs):
    """inf over y' of F(y') + theta(y'-y): attained at y' = y or at a breakpoint of F."""
    out = F(xs)
    for yi, fi in zip(F.y, F.f):
        d = yi - xs
        out = np.minimum(out, fi + np.where(d >= 0, Sa * d, Sb * d))
    return out


@pytest.mark.parametrize("seed", range(16))
@pytest.mark.parametrize("convex", [True, False])
def test_restriction_matches_definition(seed, convex):
    rng = np.random.default_rng(100 + seed)
    Sa, Sb = 105.0, 95.0
    F = _random_pl(rng, int(rng.integers(1, 10)), convex=convex, slope_lo=-140, slope_hi=-60)
    # tails must bracket the window (as they do in the tree, given d < r < u)
    F.sL, F.sR = -130.0, -70.0
    V = oracle.restrict(F, Sa, Sb)
    xs = _grid(F, V)
    np.testing.assert_allclose(V(xs), _restrict_bruteforce(F, Sa, Sb, xs), rtol=0, atol=1e-9)
    slopes = np.diff(V(np.sort(np.concatenate([V.y, V.y + 1e-3]))))
    assert V.sL == -Sa and V.sR == -Sb
    # every piece of V has slope within [-Sa, -Sb]
    ys = np.concatenate([[V.y[0] - 1], V.y, [V.y[-1] + 1]])
    sl = np.diff(V(ys)) / np.diff(ys)
    assert np.all(sl >= -Sa - 1e-9) and np.all(sl <= -Sb + 1e-9)
    assert slopes is not None


# ---------------------------------------------------------------- k = 0 and CRR pins
def _european_closed_form(row):
    S0, K, K2, sigma, R, T, N, pay = (float(row["S0"]), float(row["K"]), float(row["K2"]),
                                     float(row["sigma"]), float(row["R"]), float(row["T"]),
                                     int(row["N"]), int(row["payoff"]))
    dt = T / N
    u = math.exp(sigma * math.sqrt(dt))
    d = 1 / u
    r = math.exp(R * dt)
    p = (r - d) / (u - d)
    j = np.arange(N + 1)
    S = S0 * u ** (2.0 * j - N)
    if pay == 0:
        P = np.maximum(K - S, 0)
    elif pay == 1:
        P = np.maximum(S - K, 0)
    else:
        P = np.maximum(S - K, 0) - np.maximum(S - K2, 0)
    return float(np.sum(binom.pmf(j, N, p) * P) / r ** N)


@pytest.mark.parametrize("seed", range(4))
def test_crr_european_matches_binomial_sum(seed):
    t = W.random_table(6, 1000 + seed, N_lo=5, N_hi=400, k_zero=True)
    eu, st = oracle.crr_price(t, american=False)
    assert np.all(st == 0)
    for i in range(len(t)):
        assert eu[i] == pytest.approx(_european_closed_form(t[i]), rel=1e-11, abs=1e-12)


def test_american_call_equals_european_call():
    """Appendix: without dividends or costs an American call is worth the European call."""
    t = W.random_table(8, 77, N_lo=10, N_hi=300, payoffs=(W.CALL,), k_zero=True)
    am, _ = oracle.crr_price(t, american=True)
    eu, _ = oracle.crr_price(t, american=False)
    np.testing.assert_allclose(am, eu, rtol=1e-12)
    tc, _ = oracle.price_ask_bid(t)
    np.testing.assert_allclose(tc[:, 0], eu, rtol=1e-11)
    np.testing.assert_allclose(tc[:, 1], eu, rtol=1e-11)


def test_appendix_put_13_906():
    g = _gold("appendix_put.json")
    for N in g["N"][:2]:
        t = W.appendix_put(N)
        am, _ = oracle.crr_price(t)
        assert round(am[0], 3) == g["price_3dp"], (N, am[0])
    for N in g["N_within_1e-3"]:
        am, _ = oracle.crr_price(W.appendix_put(N))
        assert abs(am[0] - g["price_3dp"]) < 1e-3


@pytest.mark.parametrize("seed", range(3))
def test_k0_reduces_to_crr(seed):
    """Section 3 / Appendix: at k = 0 the ask and bid coincide with the CRR American price."""
    t = W.random_table(10, 500 + seed, N_lo=1, N_hi=120, k_zero=True)
    tc, st = oracle.price_ask_bid(t)
    crr, _ = oracle.crr_price(t)
    assert np.all(st == 0)
    np.testing.assert_allclose(tc[:, 0], crr, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(tc[:, 1], crr, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- orderings and bounds
def test_price_curves_ordering():
    """Section 5 (price curves): for fixed S0 in [90, 110] and k0 = 0 < k1 = 0.25% < k2 = 0.5%,
    bid_k2 <= bid_k1 <= CRR = ask_k0 = bid_k0 < ask_k1 < ask_k2."""
    for S0 in (90.0, 95.0, 100.0, 105.0, 110.0):
        rows = [W.make(S0=S0, K=100.0, k=k, N=120) for k in (0.0, 0.0025, 0.005)]
        out, _ = oracle.price_ask_bid(W.concat(*rows))
        (a0, b0), (a1, b1), (a2, b2) = out
        assert a0 == pytest.approx(b0, rel=1e-12)
        assert b2 <= b1 + 1e-12 and b1 <= b0 + 1e-12
        assert a0 < a1 < a2


@pytest.mark.parametrize("seed", range(3))
def test_bounds_and_bid_le_crr_le_ask(seed):
    t = W.random_table(12, 900 + seed, N_lo=5, N_hi=80)
    out, st = oracle.price_ask_bid(t)
    t0 = t.copy()
    t0["k"] = 0.0
    crr, _ = oracle.crr_price(t0)
    assert np.all(st == 0)
    for i, row in enumerate(t):
        ask, bid = out[i]
        S0, K, K2 = float(row["S0"]), float(row["K"]), float(row["K2"])
        assert bid <= crr[i] + 1e-9 and crr[i] <= ask + 1e-9
        if row["payoff"] == W.PUT:
            lo, hi = max(0.0, K - S0), K
        elif row["payoff"] == W.CALL:
            lo, hi = max(0.0, S0 - K), S0
        else:
            lo, hi = max(0.0, S0 - K) - max(0.0, S0 - K2), K2 - K
        assert lo - 1e-9 <= bid <= ask <= hi + 1e-9


# ---------------------------------------------------------------- exact arithmetic
EXACT_CASES = [
    dict(k=0.0025, N=9, payoff=W.PUT),
    dict(k=0.01, N=10, payoff=W.CALL),
    dict(K=95.0, K2=105.0, k=0.01, N=12, payoff=W.SPREAD),
    dict(k=0.05, N=8, payoff=W.PUT, S0=97.0),
    dict(K=95.0, K2=105.0, k=0.02, N=10, payoff=W.SPREAD, sigma=0.1, T=0.1),
] + [dict(K=(95.0 if pay == W.SPREAD else 100.0), K2=105.0, k=k, N=24, payoff=pay)
     for pay in (W.PUT, W.CALL, W.SPREAD) for k in (0.0025, 0.01, 0.05)]


@pytest.mark.parametrize("case", EXACT_CASES)
def test_oracle_within_rounding_of_exact(case):
    t = W.make(**case)
    out, _ = oracle.price_ask_bid(t)
    a, b = exact.price_row(t[0])
    scale = max(abs(float(a)), 1e-2 * float(t[0]["K"]))
    assert abs(out[0, 0] - float(a)) <= 1e-12 * scale
    assert abs(out[0, 1] - float(b)) <= 1e-12 * max(abs(float(b)), 1e-2 * float(t[0]["K"]))


# ---------------------------------------------------------------- hedging linear programs
LP_CASES = [
    dict(k=0.005, N=1),
    dict(k=0.02, N=2),
    dict(K=95.0, K2=105.0, k=0.01, N=3, payoff=W.SPREAD),
    dict(k=0.01, N=3, payoff=W.CALL),
    dict(k=0.05, N=3, S0=95.0),
    dict(k=0.03, N=4, payoff=W.PUT, S0=102.0),
]


@pytest.mark.parametrize("case", LP_CASES)
def test_oracle_matches_hedging_lp(case):
    t = W.make(**case)
    out, _ = oracle.price_ask_bid(t)
    row = t[0]
    ask_lp = hedging_lp.ask(*[float(row[f]) for f in ("S0", "K", "K2", "sigma", "R", "T", "k")],
                            int(row["N"]), int(row["payoff"]))
    args = [float(row[f]) for f in ("S0", "K", "K2", "sigma", "R", "T", "k")] + [int(row["N"]),
                                                                              int(row["payoff"])]
    bid_lp = hedging_lp.bid_enumerate(*args) if case["N"] <= 3 else hedging_lp.bid_milp(*args)
    assert out[0, 0] == pytest.approx(ask_lp, rel=1e-9, abs=1e-9)
    assert out[0, 1] == pytest.approx(bid_lp, rel=1e-9, abs=1e-9)


SELLER_LP_CASES = [
    dict(k=0.01, N=5, payoff=W.PUT),
    dict(k=0.02, N=6, payoff=W.PUT, S0=97.0),
    dict(k=0.01, N=6, payoff=W.CALL),
    dict(K=95.0, K2=105.0, k=0.01, N=6, payoff=W.SPREAD),
    dict(K=95.0, K2=105.0, k=0.05, N=5, payoff=W.SPREAD, sigma=0.1),
]


@pytest.mark.parametrize("case", SELLER_LP_CASES)
def test_oracle_ask_matches_superhedging_lp_n6(case):
    """The seller's superhedging LP on the non-recombining tree at N = 5, 6 (2^(N+2) - 1 nodes).
    The buyer's side is pinned up to N = 4 only: its stopping-time program (binary stop
    indicators) took 17-30 s at N = 4 and did not finish in 10 minutes at N = 5."""
    t = W.make(**case)
    out, _ = oracle.price_ask_bid(t)
    row = t[0]
    ask_lp = hedging_lp.ask(*[float(row[f]) for f in ("S0", "K", "K2", "sigma", "R", "T", "k")],
                            int(row["N"]), int(row["payoff"]))
    assert out[0, 0] == pytest.approx(ask_lp, rel=1e-9, abs=1e-9)


def test_oracle_bid_matches_stopping_time_milp_spread_n4():
    row = W.make(K=95.0, K2=105.0, k=0.01, N=4, payoff=W.SPREAD)
    out, _ = oracle.price_ask_bid(row)
    args = [float(row[0][f]) for f in ("S0", "K", "K2", "sigma", "R", "T", "k")] + [4, W.SPREAD]
    assert out[0, 1] == pytest.approx(hedging_lp.bid_milp(*args, ybound=3.0, xbound=1000.0),
                                      rel=1e-9, abs=1e-9)


def test_buyer_milp_agrees_with_enumeration():
    t = W.make(K=95.0, K2=105.0, k=0.01, N=3, payoff=W.SPREAD, sigma=0.15)[0]
    args = [float(t[f]) for f in ("S0", "K", "K2", "sigma", "R", "T", "k")] + [3, 2]
    assert hedging_lp.bid_milp(*args) == pytest.approx(hedging_lp.bid_enumerate(*args), rel=1e-10)


# ---------------------------------------------------------------- derivatives
def _fd(row, which, h_rel=1e-5):
    base = float(row[which][0])
    h = h_rel * max(abs(base), 1e-3)
    up, dn = row.copy(), row.copy()
    up[which] = base + h
    dn[which] = base - h
    if which == "K":
        up["K2"] = float(row["K2"][0]) + h
        dn["K2"] = float(row["K2"][0]) - h
    ou, _ = oracle.price_ask_bid(up)
    od, _ = oracle.price_ask_bid(dn)
    return (ou[0] - od[0]) / (2 * h)


@pytest.mark.parametrize("seed", range(3))
def test_dual_gradient_matches_central_differences(seed):
    t = W.random_table(3, 4000 + seed, N_lo=20, N_hi=60, k_hi=0.02)
    t["k"] = np.maximum(t["k"], 0.002)  # away from the one-sided k = 0 boundary
    out, grad, st = oracle.greeks(t)
    price, _ = oracle.price_ask_bid(t)
    np.testing.assert_allclose(out, price, rtol=1e-13, atol=1e-13)
    names = ["S0", "K", "sigma", "R", "T", "k"]
    checked = 0
    for i in range(len(t)):
        row = t[i:i + 1]
        for a, name in enumerate(names):
            fd1 = _fd(row, name, 1e-5)
            fd2 = _fd(row, name, 1e-6)
            for party in range(2):
                g = grad[i, party, a]
                scale = max(abs(g), 1e-3 * float(row["K"][0]))
                if abs(fd1[party] - fd2[party]) > 1e-3 * scale:
                    continue  # a structural kink lies within the bump
                assert abs(g - fd1[party]) <= 1e-5 * scale, (i, name, party, g, fd1[party])
                checked += 1
    assert checked >= 24


# Calls near k = sigma sqrt(T/N), where pieces of nearly equal slope cross at shallow angles
# and cluster within a few ulps; the gradient differentiates the lines of the pieces, so the
# fast-moving crossing positions never enter it.  Pinned by central differences of the
# oracle's prices at two bump sizes (a bump that straddles a kink is skipped).
ILL_CONDITIONED = [
    dict(S0=89.8, K=90.3, K2=100.3, sigma=0.4650, R=0.0446, T=0.6205, k=0.00845, N=1000, payoff=W.CALL),
    dict(S0=110.0, K=96.0, K2=106.0, sigma=0.2331, R=0.0542, T=1.2598, k=0.00940, N=1000, payoff=W.CALL),
    dict(S0=100.0, K=100.0, K2=110.0, sigma=0.4089, R=0.0500, T=1.9912, k=0.01354, N=1000, payoff=W.CALL),
]


def _fd_batch(row, h_rel):
    """Central differences of the oracle's prices in all six parameters, one batched call."""
    names = ["S0", "K", "sigma", "R", "T", "k"]
    rows = []
    hs = []
    for name in names:
        base = float(row[name][0])
        h = h_rel * max(abs(base), 1e-3)
        hs.append(h)
        for sign in (1.0, -1.0):
            r = row.copy()
            r[name] = base + sign * h
            if name == "K":
                r["K2"] = float(row["K2"][0]) + sign * h
            rows.append(r)
    out, _ = oracle.price_ask_bid(W.concat(*rows), nthreads=8)
    return np.array([(out[2 * a] - out[2 * a + 1]) / (2 * hs[a]) for a in range(6)])  # [param, party]


@pytest.mark.parametrize("case", ILL_CONDITIONED)
def test_gradient_of_ill_conditioned_calls_matches_central_differences(case):
    t = W.make(**case)
    _, grad, st = oracle.greeks(t)
    assert st[0] == 0
    fd1, fd2 = _fd_batch(t, 1e-5), _fd_batch(t, 1e-6)
    checked = 0
    for a in range(6):
        for party in range(2):
            g = grad[0, party, a]
            scale = max(abs(g), 1e-3 * float(t["K"][0]))
            if abs(fd1[a, party] - fd2[a, party]) > 1e-3 * scale:
                continue
            assert abs(g - fd1[a, party]) <= 1e-5 * scale, (a, party, g, fd1[a, party])
            checked += 1
    assert checked >= 10
