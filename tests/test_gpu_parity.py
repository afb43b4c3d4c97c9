"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerance (prices): |gpu - oracle| <= 1e-10 * max(|oracle|, 1e-2 K).  The
absolute floor keeps deep out-of-the-money bids (~0) meaningful.  The oracle
agrees with exact rational arithmetic to ~1e-15, the GPU keeps values in
future-value units and evaluates pieces by fused multiply-add, so both sit
within a few hundred ulps of the exact recursion; 1e-10 leaves room for the
ill-conditioned crossings of nearly parallel pieces.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def _ob():
    import paper_1110_2477_gb300 as ob
    return ob


def _close(got, ref, K):
    scale = np.maximum(np.abs(ref), 1e-2 * np.asarray(K)[..., None] if ref.ndim == 2 else 1e-2 * np.asarray(K))
    return np.abs(got - ref) <= RTOL * scale


def _gpu(table, plain=False):
    import torch
    ob = _ob()
    out, st = ob.price(table, plain=plain)
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy()


def _assert_parity(table, out, st, ref, rst):
    assert np.array_equal(st, rst), (st, rst)
    ok = _close(out, ref, table["K"])
    ok |= (np.isnan(out) & np.isnan(ref))
    bad = np.argwhere(~ok)
    assert bad.size == 0, [(int(i), out[i].tolist(), ref[i].tolist(), table[i]) for i, _ in bad[:5]]


def test_config1_put_n250():
    t = W.single_put_n250()
    out, st = _gpu(t)
    ref, rst = oracle.price_ask_bid(t)
    _assert_parity(t, out, st, ref, rst)
    crr, _ = oracle.crr_price(t[1:])
    assert abs(out[1, 0] - crr[0]) <= RTOL * crr[0] and abs(out[1, 1] - crr[0]) <= RTOL * crr[0]
    assert out[0, 1] <= crr[0] <= out[0, 0]


@pytest.mark.parametrize("seed", range(6))
def test_random_small_tables(seed):
    # sizes span several warp tiles per level and end in ragged tails
    t = W.random_table(48, 20000 + seed, N_lo=1, N_hi=140, k_hi=0.05 if seed % 2 else 0.02)
    out, st = _gpu(t)
    ref, rst = oracle.price_ask_bid(t, nthreads=8)
    _assert_parity(t, out, st, ref, rst)


def test_heavy_small_cases():
    # low volatility and high costs: hundreds of breakpoints per node
    t = W.concat(W.make(S0=100, K=95, K2=105, sigma=0.1, T=0.1, k=0.02, N=150, payoff=W.SPREAD),
                 W.make(S0=100, K=100, sigma=0.1, T=0.1, k=0.02, N=150, payoff=W.CALL),
                 W.make(K=95, K2=105, k=0.01, N=300, payoff=W.SPREAD),
                 W.make(S0=110, K=100, k=0.03, N=200, payoff=W.CALL))
    out, st = _gpu(t)
    ref, rst = oracle.price_ask_bid(t, nthreads=4)
    _assert_parity(t, out, st, ref, rst)


def test_k0_all_payoffs_equal_crr():
    t = W.random_table(30, 31337, N_lo=1, N_hi=200, k_zero=True)
    out, st = _gpu(t)
    ref, _ = oracle.crr_price(t)
    assert np.all(st == 0)
    for col in (0, 1):
        assert np.all(_close(out[:, col], ref, t["K"])), (out[:, col], ref)


def test_edge_cases_status():
    good = W.make(k=0.01, N=5)
    bad_N = W.make(N=0)
    bad_k = W.make(k=1.0)
    bad_sigma = W.make(sigma=0.0)
    bad_payoff = W.make()
    bad_payoff["payoff"] = 7
    bad_spread = W.make(K=100.0, K2=90.0, payoff=W.SPREAD)
    arb = W.make(R=5.0, N=2, T=1.0)  # r > u
    n1 = W.make(k=0.02, N=1)
    t = W.concat(good, bad_N, bad_k, bad_sigma, bad_payoff, bad_spread, arb, n1)
    out, st = _gpu(t)
    ref, rst = oracle.price_ask_bid(t)
    # the oracle's codes: -1 argument, -2 arbitrage; the library's are the same numbers
    assert st.tolist() == rst.tolist() == [0, -1, -1, -1, -1, -1, -2, 0]
    assert np.all(np.isnan(out[1:7]))
    _assert_parity(t[[0, 7]], out[[0, 7]], st[[0, 7]], ref[[0, 7]], rst[[0, 7]])


def test_empty_batch_is_noop():
    import torch
    ob = _ob()
    params = torch.empty(0, dtype=torch.uint8, device="cuda")
    out = torch.empty(0, dtype=torch.float64, device="cuda")
    ob.ob_price_ask_bid(params, 0, out)
    ob.ob_crr_american(params, 0, out)
    ob.ob_price_ask_bid_hedge(params, 0, out, None, None)
    ob.ob_price_ask_bid_plain(params, 0, out)
    ob.ob_price_ask_bid_wide(params, 0, out)
    ob.ob_crr_american_wide(params, 0, out)
    ob.ob_price_ask_bid_noalloc(params, 0, out)
    ob.ob_greeks(params, 0, out, out)
    torch.cuda.synchronize()


def test_batched_equals_plain_bitwise():
    t = W.random_table(64, 555, N_lo=20, N_hi=300)
    a, sa = _gpu(t, plain=False)
    b, sb = _gpu(t, plain=True)
    assert np.array_equal(sa, sb)
    assert np.array_equal(a.view(np.int64), b.view(np.int64))


def test_host_buffer_entry_matches_device():
    ob = _ob()
    t = W.random_table(40, 99, N_lo=10, N_hi=200)
    d, ds = _gpu(t)
    out = np.empty((len(t), 2), np.float64)
    st = np.empty(len(t), np.int32)
    ob.ob_price_ask_bid_host(t, out, st)
    assert np.array_equal(st, ds)
    assert np.array_equal(out.view(np.int64), d.view(np.int64))


def test_stats_count_node_updates():
    ob = _ob()
    t = W.random_table(50, 4242, N_lo=5, N_hi=100)
    _gpu(t)
    s = ob.ob_get_stats()
    assert s["options"] == len(t) and s["failed"] == 0
    assert s["node_updates"] == int(np.sum(W.node_updates(t)))
    assert s["z_points"] >= s["node_updates"]  # every node keeps >= 1 breakpoint per party... at least one


# ---------------------------------------------------------------- full-size configurations
def test_batched_4096_sampled():
    """The batched uneven workload at full size; the oracle checks a stratified sample."""
    t = W.batched_uneven()
    out, st = _gpu(t)
    assert np.all(st == 0)
    assert np.all(np.isfinite(out))
    rng = np.random.default_rng(0)
    order = np.argsort(t["N"])
    idx = np.unique(np.concatenate([order[:8], rng.choice(len(t), 10, replace=False)]))
    ref, rst = oracle.price_ask_bid(t[idx], nthreads=16)
    _assert_parity(t[idx], out[idx], st[idx], ref, rst)
    # properties at every option: bid <= CRR <= ask
    t0 = t.copy()
    t0["k"] = 0.0
    crr, _ = _ob().crr(t0)
    crr = crr.cpu().numpy()
    assert np.all(out[:, 1] <= crr * (1 + 1e-12) + 1e-12)
    assert np.all(out[:, 0] >= crr * (1 - 1e-12) - 1e-12)


def test_paper_scale_n1500_single_launches():
    t = W.paper_scale(Ns=(1500,), ks=(0.005, 0.01))
    outs = []
    for i in range(len(t)):
        o, s = _gpu(t[i:i + 1])
        assert s[0] == 0
        outs.append(o[0])
    out = np.array(outs)
    ref, rst = oracle.price_ask_bid(t, nthreads=4)
    _assert_parity(t, out, np.zeros(len(t), np.int32), ref, rst)


def test_paper_scale_large_n_properties():
    t = W.paper_scale(Ns=(3000, 6000))
    out, st = _gpu(t)
    assert np.all(st == 0)
    puts, spreads = out[0::2], out[1::2]
    for grp in (puts, spreads):
        for N_blk in range(2):
            blk = grp[3 * N_blk:3 * N_blk + 3]  # k increasing
            assert np.all(np.diff(blk[:, 0]) > 0) and np.all(np.diff(blk[:, 1]) <= 1e-12)
    ref, rst = oracle.price_ask_bid(t[:1], nthreads=1)  # N = 3000 put, k = 0.0025
    _assert_parity(t[:1], out[:1], st[:1], ref, rst)


def test_greeks_config_puts_sampled():
    t = W.greeks_puts()
    out, st = _gpu(t)
    assert np.all(st == 0)
    idx = np.arange(0, len(t), 128)
    ref, rst = oracle.price_ask_bid(t[idx], nthreads=8)
    _assert_parity(t[idx], out[idx], st[idx], ref, rst)


# ---------------------------------------------------------------- plain CRR kernel
@pytest.mark.parametrize("seed", range(3))
def test_crr_kernel_random(seed):
    t = W.random_table(200, 600 + seed, N_lo=1, N_hi=2500, k_zero=True)
    got, st = _ob().crr(t)
    got, st = got.cpu().numpy(), st.cpu().numpy()
    ref, rst = oracle.crr_price(t, nthreads=8)
    assert np.array_equal(st, rst)
    assert np.all(_close(got, ref, t["K"])), np.max(np.abs(got - ref) / np.maximum(ref, 1))


def test_crr_65536_sampled_and_appendix_put():
    t = W.crr_puts()
    got, st = _ob().crr(t)
    got, st = got.cpu().numpy(), st.cpu().numpy()
    assert np.all(st == 0)
    idx = np.arange(0, len(t), 4096)
    ref, _ = oracle.crr_price(t[idx], nthreads=8)
    assert np.all(_close(got[idx], ref, t["K"][idx]))
    big = W.appendix_put(20000)
    g, s = _ob().crr(big)
    g = g.cpu().numpy()
    r, _ = oracle.crr_price(big)
    assert s.cpu().numpy()[0] == 0 and abs(g[0] - r[0]) <= RTOL * r[0]
    assert round(float(g[0]), 3) == 13.906


# ---------------------------------------------------------------- scratch limits (subprocess: the pool is per process)
_CHILD = r"""
import sys, json, numpy as np, torch
sys.path.insert(0, %(root)r)
import workloads as W, paper_1110_2477_gb300 as ob
t = W.concat(W.make(K=95, K2=105, sigma=0.1, T=0.1, k=0.02, N=1000, payoff=W.SPREAD),
             W.random_table(40, 77, N_lo=50, N_hi=600))
out, st = ob.price(t)
torch.cuda.synchronize()
print(json.dumps({"out": out.cpu().numpy().tolist(), "st": st.cpu().numpy().tolist(),
                  "stats": ob.ob_get_stats()}))
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
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_capacity_retry_and_exhaustion():
    """Small per-warp slices force follow-up launches with larger slices (same results);
    a pool too small for an option yields OB_ERR_CAPACITY for it, the others complete."""
    base = _child({})
    small = _child({"OB_SM_KB": "2048"})  # 2 MiB of first-tier scratch per CTA
    assert small["stats"]["retried"] > 0
    assert small["st"] == base["st"] == [0] * len(base["st"])
    assert np.array_equal(np.array(small["out"]).view(np.int64), np.array(base["out"]).view(np.int64))
    tiny = _child({"OB_POOL_MB": "3"})
    st = np.array(tiny["st"])
    assert st[0] == -3 and np.isnan(tiny["out"][0][0])
    ok = st == 0
    assert ok.sum() >= 1
    np.testing.assert_array_equal(np.array(tiny["out"])[ok], np.array(base["out"])[ok])


# ---------------------------------------------------------------- graphs, team widths, autotuner
def test_team_widths_and_on_chip_step_give_bitwise_equal_prices():
    """Every team width, and the fused level step with w in shared memory (all that fits,
    and a small chunk so that nodes and chunks fall back to the global scratch), price the
    same bits."""
    ob = _ob()
    t = W.concat(W.random_table(96, 4711, N_lo=20, N_hi=400),
                 W.make(S0=100, K=100, sigma=0.1, T=0.1, k=0.02, N=300, payoff=W.CALL))
    try:
        res = []
        for tw, chip in ((16, 0), (12, 0), (8, 0), (4, 0), (16, -1), (8, -1), (16, 300)):
            ob.ob_configure(team_warps=tw, use_graphs=0, chip_points=chip)
            out, st = _gpu(t)
            s = ob.ob_get_stats()
            assert s["team_warps"] == tw
            assert (s["chip_points"] > 0) == (chip != 0)
            res.append((out, st))
        for out, st in res[1:]:
            assert np.array_equal(st, res[0][1])
            assert np.array_equal(out.view(np.int64), res[0][0].view(np.int64))
    finally:
        ob.ob_configure(team_warps=16, use_graphs=1, chip_points=0)


def test_graph_capture_then_replay_reads_current_inputs():
    """The second call with the same buffers replays the captured graph; it must price
    the records the buffer holds now, and match direct launches bit for bit."""
    import torch
    ob = _ob()
    t1 = W.random_table(64, 808, N_lo=10, N_hi=300)
    t2 = W.random_table(64, 909, N_lo=10, N_hi=300)
    dev = ob.to_device(t1)
    out = torch.empty((64, 2), dtype=torch.float64, device="cuda")
    st = torch.empty(64, dtype=torch.int32, device="cuda")
    try:
        ob.ob_configure(use_graphs=1)
        ob.ob_price_ask_bid(dev, 64, out, st)
        torch.cuda.synchronize()
        assert ob.ob_get_stats()["graph"] == 1
        r1 = out.cpu().numpy().copy()
        dev.copy_(ob.to_device(t2))
        ob.ob_price_ask_bid(dev, 64, out, st)
        torch.cuda.synchronize()
        s = ob.ob_get_stats()
        assert s["graph"] == 2 and s["options"] == 64
        r2 = out.cpu().numpy().copy()
        ob.ob_configure(use_graphs=0)
        d1, _ = _gpu(t1)
        d2, _ = _gpu(t2)
        assert ob.ob_get_stats()["graph"] == 0
        assert np.array_equal(r1.view(np.int64), d1.view(np.int64))
        assert np.array_equal(r2.view(np.int64), d2.view(np.int64))
    finally:
        ob.ob_configure(team_warps=16, use_graphs=1, chip_points=0)


def test_autotune_keeps_a_valid_configuration_and_prices_match_oracle():
    ob = _ob()
    t = W.random_table(200, 2024, N_lo=50, N_hi=500)
    before, _ = _gpu(t)
    try:
        tw, chip, ms = ob.autotune(t, sample=100)
        assert tw in (4, 8, 12, 16) and all(v > 0 for v in ms.values())
        after, st = _gpu(t)
        s = ob.ob_get_stats()
        assert s["team_warps"] == tw and s["chip_points"] == chip
        chosen = "%d+chip" % tw if chip else ("16-whole" if tw == 16 and not s["half_teams"] else "%d" % tw)
        assert len(ms) == 7 and ms[chosen] <= min(ms.values()) / 0.99
        assert np.array_equal(before.view(np.int64), after.view(np.int64))
        idx = np.arange(0, len(t), 25)
        ref, rst = oracle.price_ask_bid(t[idx], nthreads=8)
        _assert_parity(t[idx], after[idx], st[idx], ref, rst)
    finally:
        ob.ob_configure(team_warps=16, use_graphs=1, chip_points=0)


# ---------------------------------------------------------------- whole-GPU form (large single options)
def _wide(table):
    import torch
    out, st = _ob().price(table, wide=True)
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy()


def test_wide_equals_batched_bitwise_with_edge_cases():
    """Every SM on one option at a time: same bits and statuses as the batched form,
    including N = 1, 2 (most CTAs own no node), invalid records and an arbitrage tree."""
    t = W.concat(W.random_table(12, 5150, N_lo=1, N_hi=300), W.make(k=0.01, N=1), W.make(k=0.01, N=2),
                 W.make(N=0), W.make(R=5.0, N=2, T=1.0),
                 W.make(S0=100, K=100, sigma=0.1, T=0.1, k=0.02, N=200, payoff=W.CALL))
    a, sa = _gpu(t)
    b, sb = _wide(t)
    assert np.array_equal(sa, sb)
    ok = sa == 0
    assert np.array_equal(a[ok].view(np.int64), b[ok].view(np.int64))
    assert np.all(np.isnan(b[~ok]))


def test_wide_paper_scale_matches_oracle_and_batched():
    t = W.paper_scale(Ns=(1500,), ks=(0.005,))
    b, sb = _wide(t)
    assert np.all(sb == 0)
    s = _ob().ob_get_stats()
    a, sa = _gpu(t)
    s2 = _ob().ob_get_stats()
    assert np.array_equal(a.view(np.int64), b.view(np.int64))
    assert s["node_updates"] == s2["node_updates"]
    # the trapezoid rounds recompute halo columns and publish every D-th level only
    for k in ("u_points", "w_points", "z_points"):
        assert s[k] >= s2[k], k
    assert s["max_level_points"] <= s2["max_level_points"]
    ref, rst = oracle.price_ask_bid(t, nthreads=2)
    _assert_parity(t, b, sb, ref, rst)


# ---------------------------------------------------------------- price curves at scale
def test_price_curves_ordering_at_scale():
    """Section 5's price curves at N = 1500 for 41 values of S0 in [90, 110]: at every S0,
    bid(0.5%) <= bid(0.25%) <= CRR = ask(0) = bid(0) < ask(0.25%) < ask(0.5%); the k = 0 prices
    equal the CRR kernel's; a sample matches the oracle."""
    ks = (0.0, 0.0025, 0.005)
    t = W.price_curves(ks=ks, N=1500)
    out, st = _gpu(t)
    assert np.all(st == 0)
    o = out.reshape(-1, len(ks), 2)
    ask, bid = o[..., 0], o[..., 1]
    crr, _ = _ob().crr(t[0::3])
    crr = crr.cpu().numpy()
    assert np.all(np.abs(ask[:, 0] - bid[:, 0]) <= 1e-12 * ask[:, 0])
    assert np.all(np.abs(ask[:, 0] - crr) <= RTOL * np.maximum(crr, 1.0))
    assert np.all(bid[:, 2] <= bid[:, 1] + 1e-12) and np.all(bid[:, 1] <= bid[:, 0] + 1e-12)
    assert np.all(ask[:, 0] < ask[:, 1]) and np.all(ask[:, 1] < ask[:, 2])
    idx = np.array([1, 5, 61, 119, 122])
    ref, rst = oracle.price_ask_bid(t[idx], nthreads=5)
    _assert_parity(t[idx], out[idx], st[idx], ref, rst)


# ---------------------------------------------------------------- CRR on the whole GPU
def test_crr_wide_equals_crr_kernel_bitwise():
    """Trapezoid tiles of 64 levels over every SM give the same bits as the warp kernel,
    for N below and above a tile, above the warp kernel's shared-memory size, and for the
    invalid and arbitrage records."""
    t = W.concat(W.random_table(40, 6100, N_lo=1, N_hi=3000, k_zero=True), W.make(k=0.0, N=1),
                 W.make(k=0.0, N=64), W.make(k=0.0, N=65), W.make(N=0), W.make(R=5.0, N=2, T=1.0),
                 W.make(k=0.0, N=2400, payoff=W.SPREAD, K=95.0, K2=105.0))
    a, sa = _ob().crr(t)
    b, sb = _ob().crr(t, wide=True)
    a, sa, b, sb = a.cpu().numpy(), sa.cpu().numpy(), b.cpu().numpy(), sb.cpu().numpy()
    assert np.array_equal(sa, sb)
    ok = sa == 0
    assert np.array_equal(a[ok].view(np.int64), b[ok].view(np.int64))
    assert np.all(np.isnan(b[~ok]))


def test_crr_wide_appendix_put_large_n():
    """The Appendix put at N = 20000 and 40000 on the whole GPU: 13.906, and the oracle."""
    t = W.concat(W.appendix_put(20000), W.appendix_put(40000))
    g, s = _ob().crr(t, wide=True)
    g, s = g.cpu().numpy(), s.cpu().numpy()
    ref, _ = oracle.crr_price(t, nthreads=2)
    assert np.all(s == 0)
    assert np.all(np.abs(g - ref) <= RTOL * ref)
    assert [round(float(x), 3) for x in g] == [13.906, 13.906]


def test_wide_with_costs_at_n_10000_and_20000():
    """Single options with costs beyond the paper's sizes on the whole GPU (N = 10000 and
    20000): every status is OK, and the prices keep Section 5's ordering (bid <= the CRR
    price <= ask, the ask rising and the bid falling with k, equal at k = 0)."""
    recs = []
    for N in (10000, 20000):
        for k in (0.0, 0.0025, 0.005):
            recs.append(W.make(k=k, N=N))
        recs.append(W.make(K=95.0, K2=105.0, k=0.0025, N=N, payoff=W.SPREAD))
    t = W.concat(*recs)
    out, st = _ob().price(t, wide=True)
    crr, cst = _ob().crr(t)
    out, st, crr = out.cpu().numpy(), st.cpu().numpy(), crr.cpu().numpy()
    assert np.all(st == 0) and np.all(cst.cpu().numpy() == 0)
    for b in (0, 4):
        p0, p1, p2 = out[b], out[b + 1], out[b + 2]
        assert abs(p0[0] - p0[1]) <= 1e-9 * p0[0] and abs(p0[0] - crr[b]) <= 1e-9 * crr[b]
        assert p2[1] <= p1[1] <= crr[b + 1] <= p1[0] <= p2[0]
        assert p1[0] > p0[0] and p1[1] < p0[1]
        sp = out[b + 3]
        assert sp[1] <= crr[b + 3] <= sp[0] and 0.0 <= sp[1] and sp[0] <= 10.0


_SPLIT_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, %(root)r)
import workloads as W, paper_1110_2477_gb300 as ob
t = W.random_table(600, 8181, N_lo=2, N_hi=900)
out, st = ob.price(t)
torch.cuda.synchronize()
np.save(%(npy)r, np.concatenate([out.cpu().numpy().reshape(-1), st.cpu().numpy().astype(np.float64)]))
"""


def test_split_factor_gives_the_same_bits(tmp_path):
    """The point where 16-warp CTAs split into two 8-warp teams (OB_SPLIT_FACTOR: off, the
    default, everything on halves) changes which team prices an option, never the result."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = []
    for sf in ("0", "0.04", "1000"):
        npy = str(tmp_path / ("s%s.npy" % sf))
        env = dict(os.environ, OB_SPLIT_FACTOR=sf)
        r = subprocess.run([sys.executable, "-c", _SPLIT_CHILD % {"root": root, "npy": npy}], env=env,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        res.append(np.load(npy))
    assert np.all(res[0][-600:] == 0)
    for x in res[1:]:
        assert np.array_equal(x.view(np.int64), res[0].view(np.int64))


_WIDE_MODE_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, %(root)r)
import workloads as W, paper_1110_2477_gb300 as ob
t = W.concat(W.random_table(12, 9393, N_lo=40, N_hi=700, payoffs=(W.CALL, W.SPREAD), k_hi=0.05),
             W.make(K=95.0, K2=105.0, k=0.01, N=1500, payoff=W.SPREAD),
             W.make(k=0.02, N=900, sigma=0.1, payoff=W.CALL), W.make(k=0.005, N=300))
out, st = ob.price(t, wide=True)
ref, rst = ob.price(t)
torch.cuda.synchronize()
np.save(%(npy)r, np.concatenate([out.cpu().numpy().reshape(-1), ref.cpu().numpy().reshape(-1),
                                  st.cpu().numpy().astype(np.float64), rst.cpu().numpy().astype(np.float64)]))
"""


def test_wide_node_split_gives_the_same_bits(tmp_path):
    """The whole-GPU form with nodes split over the CTAs at the quantiles of the merged points
    (OB_WIDE_SPLIT_X=-1: every level of every call and spread), with the default choice (calls
    and spreads with k > 6 sigma sqrt(dt), on levels whose largest node outgrows a share), and
    with none (shares of whole nodes) prices bit for bit as the batched form."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    n = 15
    for x in ("-1", "6", "1e9"):
        npy = str(tmp_path / ("w%s.npy" % x))
        env = dict(os.environ, OB_WIDE_SPLIT_X=x)
        r = subprocess.run([sys.executable, "-c", _WIDE_MODE_CHILD % {"root": root, "npy": npy}], env=env,
                           capture_output=True, text=True, timeout=900)
        assert r.returncode == 0, r.stderr[-2000:]
        a = np.load(npy)
        wide, batched = a[:2 * n], a[2 * n:4 * n]
        st, rst = a[4 * n:5 * n], a[5 * n:]
        assert np.all(st == 0) and np.all(rst == 0), x
        assert np.array_equal(wide.view(np.int64), batched.view(np.int64)), x
