"""The hedge along a path of the tree on the GPU (ob_hedge_path) against the oracle.

  * prices: bitwise those of ob_price_ask_bid on the same records;
  * holdings: the oracle's within 1e-9 (relative to max(1, |y|)) at every level of the path,
    NaN in the same places (beyond N_i, and from the buyer's stopping level on);
  * cash: the oracle's within 1e-9 relative to max(|x|, S0); the two carry it in different
    units (the kernel in future-value units, the oracle in time-t money, growing by r a
    level), so they round differently over N levels of trades of size up to S |dy|;
  * the buyer's stopping level: the oracle's;
  * paths: random, all up, all down, alternating; rows longer than N_i; N = 1;
  * a batch above the cost-ordering limit (8192 options: taken in index order);
  * an option with N_i > stride, and one that fails its checks, carry NaN and their status;
  * the paper's option sizes (N = 1500) on a sample of paths;
  * the benchmark's path workload in its launch configuration, sampled;
  * small first-tier slices (the follow-up launch, same bits) and a pool too small for one
    option (OB_ERR_CAPACITY for it, the others complete).
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _gpu(table, moves):
    import torch

    import paper_1110_2477_gb300 as ob
    out, hold, cash, stop, st = ob.hedge_path(table, moves)
    ref_out, ref_st = ob.price(table)
    torch.cuda.synchronize()
    return (out.cpu().numpy(), hold.cpu().numpy(), cash.cpu().numpy(), stop.cpu().numpy(), st.cpu().numpy(),
            ref_out.cpu().numpy(), ref_st.cpu().numpy())


def _close_cash(g, o, S0):
    fin = ~np.isnan(o)
    assert np.array_equal(np.isnan(g), ~fin)
    scale = np.maximum(np.abs(o), S0)
    err = np.abs(g - o)[fin] / scale[fin]
    assert err.max(initial=0.0) <= 1e-9, err.max()


def _check(table, moves, nthreads=8):
    out, hold, cash, stop, st, ref_out, ref_st = _gpu(table, moves)
    assert np.array_equal(st, ref_st)
    assert np.array_equal(out.view(np.int64), ref_out.view(np.int64))
    oh, oc, ostop, ost = oracle.hedge_path(table, moves, nthreads=nthreads)
    assert np.array_equal(st, ost)
    ok = st == 0
    assert np.array_equal(stop[ok], ostop[ok])
    assert np.all(stop[~ok] == -1)
    assert np.all(np.isnan(hold[~ok])) and np.all(np.isnan(cash[~ok]))
    _close_cash(cash[ok], oc[ok], table["S0"][ok][:, None, None])
    g, o = hold[ok], oh[ok]
    assert np.array_equal(np.isnan(g), np.isnan(o))
    fin = ~np.isnan(o)
    err = np.abs(g[fin] - o[fin]) / np.maximum(1.0, np.abs(o[fin]))
    assert err.max(initial=0.0) <= 1e-9, err.max()
    return out, hold, stop, st


def test_random_paths_mixed_payoffs():
    t = W.random_table(40, 7070, N_lo=2, N_hi=260)
    rng = np.random.default_rng(17)
    mv = rng.integers(0, 2, (len(t), int(t["N"].max()) + 3)).astype(np.int8)
    _, hold, stop, _ = _check(t, mv)
    assert np.any(stop >= 0)  # some buyers stop on their paths


@pytest.mark.parametrize("kind", ["up", "down", "alternate"])
def test_extreme_paths(kind):
    t = W.concat(W.make(N=120, payoff=W.PUT, k=0.004), W.make(N=97, payoff=W.CALL, k=0.01, R=0.03),
                 W.make(N=150, payoff=W.SPREAD, K2=110.0, k=0.002, sigma=0.3), W.make(N=1, k=0.01),
                 W.make(N=64, payoff=W.PUT, k=0.0, S0=80.0))
    S = int(t["N"].max())
    if kind == "up":
        mv = np.ones((len(t), S), np.int8)
    elif kind == "down":
        mv = np.zeros((len(t), S), np.int8)
    else:
        mv = np.tile(np.arange(S) % 2, (len(t), 1)).astype(np.int8)
    _check(t, mv)


def test_no_costs_holdings_are_the_oracle_crr_deltas():
    t = W.random_table(24, 8181, N_lo=2, N_hi=200, k_zero=True)
    mv = np.random.default_rng(5).integers(0, 2, (len(t), int(t["N"].max()))).astype(np.int8)
    _check(t, mv)


def test_short_rows_and_bad_options():
    t = W.concat(W.make(N=50), W.make(N=30), W.make(N=40, sigma=-1.0), W.make(N=40))
    mv = np.random.default_rng(9).integers(0, 2, (len(t), 40)).astype(np.int8)
    out, hold, cash, stop, st, ref_out, ref_st = _gpu(t, mv)
    assert st[0] == -1 and np.all(np.isnan(out[0])) and np.all(np.isnan(hold[0])) and stop[0] == -1
    assert np.all(np.isnan(cash[0])) and np.all(np.isnan(cash[2]))
    assert st[2] == -1 and np.all(np.isnan(out[2])) and np.all(np.isnan(hold[2]))
    assert st[1] == 0 and st[3] == 0
    assert np.all(np.isnan(hold[1, 31:]))
    oh, oc, ostop, ost = oracle.hedge_path(t[[1, 3]], mv[[1, 3]])
    for gi, oi in ((1, 0), (3, 1)):
        assert np.array_equal(out[gi].view(np.int64), ref_out[gi].view(np.int64))
        assert stop[gi] == ostop[oi]
        g, o = hold[gi], oh[oi]
        assert np.array_equal(np.isnan(g), np.isnan(o))
        fin = ~np.isnan(o)
        assert np.all(np.abs(g[fin] - o[fin]) <= 1e-9 * np.maximum(1.0, np.abs(o[fin])))
        _close_cash(cash[gi], oc[oi], t["S0"][gi])


def test_batch_above_the_ordering_limit():
    t = W.random_table(8200, 9090, N_lo=1, N_hi=6)
    mv = np.random.default_rng(31).integers(0, 2, (len(t), 6)).astype(np.int8)
    _check(t, mv)


def test_empty_batch():
    import torch

    import paper_1110_2477_gb300 as ob
    p = torch.empty((0, 8), dtype=torch.float64, device="cuda")
    mv = torch.zeros((0, 4), dtype=torch.int8, device="cuda")
    out = torch.empty((0, 2), dtype=torch.float64, device="cuda")
    hold = torch.empty((0, 5, 2), dtype=torch.float64, device="cuda")
    stop = torch.empty(0, dtype=torch.int32, device="cuda")
    ob.ob_hedge_path(p, 0, mv, 4, out, hold, hold, stop)
    torch.cuda.synchronize()


def test_paper_size_sample():
    t = W.concat(W.make(N=1500, payoff=W.PUT, k=0.005), W.make(N=1500, payoff=W.CALL, k=0.0025),
                 W.make(N=1500, payoff=W.SPREAD, K2=110.0, k=0.005))
    mv = np.random.default_rng(23).integers(0, 2, (len(t), 1500)).astype(np.int8)
    _check(t, mv, nthreads=3)


def test_cash_is_optional():
    import torch

    import paper_1110_2477_gb300 as ob
    t = W.concat(W.make(N=80, k=0.01), W.make(N=60, payoff=W.CALL, k=0.004))
    mv = np.random.default_rng(12).integers(0, 2, (len(t), 80)).astype(np.int8)
    dev = ob.to_device(t)
    m = torch.as_tensor(mv).cuda()
    out = torch.empty((2, 2), dtype=torch.float64, device="cuda")
    hold = torch.empty((2, 81, 2), dtype=torch.float64, device="cuda")
    stop = torch.empty(2, dtype=torch.int32, device="cuda")
    ob.ob_hedge_path(dev, 2, m, 80, out, hold, None, stop)
    out2, hold2, cash2, stop2, st2 = ob.hedge_path(t, mv)
    torch.cuda.synchronize()
    assert torch.equal(out.view(torch.int64), out2.view(torch.int64))
    assert torch.equal(torch.nan_to_num(hold, 7.0), torch.nan_to_num(hold2, 7.0))
    assert torch.equal(stop, stop2)


def test_path_workload_full_launch_sampled():
    """The benchmark's path workload in its own launch configuration (1024 puts, N = 1000,
    one random path each, seed 8), 16 sampled options against the oracle."""
    t = W.greeks_puts()
    mv = np.random.default_rng(8).integers(0, 2, (len(t), int(t["N"].max()))).astype(np.int8)
    out, hold, cash, stop, st, ref_out, ref_st = _gpu(t, mv)
    assert np.all(st == 0)
    assert np.array_equal(out.view(np.int64), ref_out.view(np.int64))
    idx = np.random.default_rng(2).choice(len(t), 16, replace=False)
    oh, oc, ostop, ost = oracle.hedge_path(t[idx], mv[idx], nthreads=8)
    assert np.all(ost == 0) and np.array_equal(stop[idx], ostop)
    g, o = hold[idx], oh
    assert np.array_equal(np.isnan(g), np.isnan(o))
    fin = ~np.isnan(o)
    assert np.all(np.abs(g[fin] - o[fin]) <= 1e-9 * np.maximum(1.0, np.abs(o[fin])))
    _close_cash(cash[idx], oc, t["S0"][idx][:, None, None])


# ---------------------------------------------------------------- scratch limits (subprocess: the pool is per process)
_CHILD = r"""
import sys, json, numpy as np, torch
sys.path.insert(0, %(root)r)
import workloads as W, paper_1110_2477_gb300 as ob
t = W.concat(W.make(K=95, K2=105, sigma=0.1, T=0.1, k=0.02, N=1000, payoff=W.SPREAD),
             W.random_table(40, 78, N_lo=50, N_hi=300))
mv = np.random.default_rng(4).integers(0, 2, (len(t), 1000)).astype(np.int8)
out, hold, cash, stop, st = ob.hedge_path(t, mv)
torch.cuda.synchronize()
print(json.dumps({"out": out.cpu().numpy().view(np.int64).tolist(),
                  "hold": hold.cpu().numpy().view(np.int64).tolist(),
                  "cash": cash.cpu().numpy().view(np.int64).tolist(),
                  "stop": stop.cpu().numpy().tolist(), "st": st.cpu().numpy().tolist()}))
"""


def _child(env_extra):
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", _CHILD % {"root": root}], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return {k: np.array(v) for k, v in json.loads(r.stdout.strip().splitlines()[-1]).items()}


def test_capacity_follow_up_launch_and_exhaustion():
    """1 MiB first-tier slices send the larger options to the follow-up launch on the whole
    pool: the same bits as with 128 MiB slices.  A 3 MiB pool is too small for the N = 1000
    spread: OB_ERR_CAPACITY and NaN for it, the others complete with the same bits."""
    base = _child({})
    assert np.all(base["st"] == 0)
    small = _child({"OB_PATH_MB": "1"})
    for k in base:
        assert np.array_equal(small[k], base[k]), k
    tiny = _child({"OB_POOL_MB": "3"})
    assert tiny["st"][0] == -3 and tiny["stop"][0] == -1
    for k in ("out", "hold", "cash"):
        assert np.all(np.isnan(tiny[k][0].view(np.float64))), k
    assert set(tiny["st"].tolist()) <= {0, -3}
    ok = tiny["st"] == 0
    assert ok.sum() >= 1
    for k in base:
        assert np.array_equal(tiny[k][ok], base[k][ok]), k
