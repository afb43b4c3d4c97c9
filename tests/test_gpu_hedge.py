"""The hedge at the root on the GPU (ob_price_ask_bid_hedge) against the oracle.

  * prices: bitwise those of ob_price_ask_bid on the same records;
  * the holding y*: the oracle's within 1e-9 (relative to max(1, |y*|)), or, where another
    breakpoint attains the same minimum to within rounding, one whose objective value is the
    oracle's minimum within 1e-12 relative;
  * the exercise flags: equal to the oracle's wherever u_0(0) and v_0(0) are not within
    rounding of each other;
  * without costs the hedge is the CRR delta at t = 0 (seller) and its negative (buyer),
    from a textbook recursion in the oracle's pin test;
  * an option that fails carries NaN.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _gpu(table):
    import torch

    import paper_1110_2477_gb300 as ob
    out, hg, st = ob.hedge(table)
    ref_out, ref_st = ob.price(table)
    torch.cuda.synchronize()
    return (out.cpu().numpy(), hg.cpu().numpy(), st.cpu().numpy(), ref_out.cpu().numpy(),
            ref_st.cpu().numpy())


def _check(table, out, hg, st, ref_out, ref_st):
    assert np.array_equal(st, ref_st)
    assert np.array_equal(out.view(np.int64), ref_out.view(np.int64))
    oh, ost = oracle.initial_hedge(table, nthreads=8)
    assert np.array_equal(st, ost)
    for i in range(len(table)):
        if st[i] != 0:
            assert np.all(np.isnan(hg[i]))
            continue
        for p in (0, 1):
            yg, yo = hg[i, p], oh[i, p]
            if abs(yg - yo) <= 1e-9 * max(1.0, abs(yo)):
                continue
            f = oracle.root_objective(table[i:i + 1], p, [yg, yo])
            assert abs(f[0] - f[1]) <= 1e-12 * max(1.0, abs(f[1])), (i, p, yg, yo, f)
        ex = oracle.root_objective(table[i:i + 1], 0, [oh[i, 0]])[0]
        assert hg[i, 2] in (0.0, 1.0) and hg[i, 3] in (0.0, 1.0)
        if hg[i, 2] != oh[i, 2] or hg[i, 3] != oh[i, 3]:
            # only a near-tie between u_0(0) and v_0(0) may flip a flag
            o = table[i]
            S0 = o["S0"]
            xi = o["K"] if o["payoff"] == W.PUT else (-o["K"] if o["payoff"] == W.CALL else
                                                       max(S0 - o["K"], 0) - max(S0 - o["K2"], 0))
            zeta = -1.0 if o["payoff"] == W.PUT else (1.0 if o["payoff"] == W.CALL else 0.0)
            u0 = xi + zeta * S0
            vb = oracle.root_objective(table[i:i + 1], 1, [oh[i, 1]])[0]
            near = (abs(u0 - ex) <= 1e-11 * max(1.0, abs(u0)) or
                    abs(-u0 - vb) <= 1e-11 * max(1.0, abs(u0)))
            assert near, (i, hg[i], oh[i], u0, ex, vb)


def test_random_table_matches_oracle():
    t = W.random_table(160, 9100, N_lo=2, N_hi=400)
    _check(t, *_gpu(t))


def test_costly_calls_and_spreads_and_edge_cases():
    t = W.concat(W.make(k=0.02, N=300, sigma=0.1, payoff=W.CALL),
                 W.make(K=95.0, K2=105.0, k=0.015, N=250, sigma=0.12, payoff=W.SPREAD),
                 W.make(S0=50.0, K=100.0, k=0.005, N=80),     # deep in the money: exercise at once
                 W.make(k=0.005, N=1),                         # one step
                 W.make(k=0.005, N=50, R=50.0),                # arbitrage: NaN
                 W.make(k=0.0, N=200, payoff=W.CALL))
    out, hg, st, ref_out, ref_st = _gpu(t)
    assert st[4] == -2 and np.all(np.isnan(hg[4]))
    assert hg[2, 2] == 1.0
    _check(t, out, hg, st, ref_out, ref_st)


def test_no_costs_hedge_is_crr_delta_on_gpu():
    from test_hedge_oracle import _crr_level1
    rng = np.random.default_rng(404)
    recs = [W.make(S0=float(rng.uniform(80, 120)), K=100.0, K2=110.0, sigma=float(rng.uniform(0.1, 0.5)),
                   R=float(rng.uniform(0.0, 0.1)), T=float(rng.uniform(0.1, 2.0)), k=0.0,
                   N=int(rng.integers(2, 300)), payoff=int(rng.integers(0, 3))) for _ in range(40)]
    t = W.concat(*recs)
    out, hg, st, _, _ = _gpu(t)
    assert np.all(st == 0)
    for i in range(len(t)):
        Vu, Vd, Su, Sd, _, _ = _crr_level1(t[i])
        delta = (Vu - Vd) / (Su - Sd)
        assert abs(hg[i, 0] - delta) <= 1e-9 * max(1.0, abs(delta)), (i, hg[i], delta)
        assert abs(hg[i, 1] + delta) <= 1e-9 * max(1.0, abs(delta)), (i, hg[i], delta)
