"""The full-size configurations against stored oracle values, element by element.

The stored values (tests/golden/*.json) were written by tests/golden/make_golden.py,
which calls only the CPU oracle.  Prices: |gpu - oracle| <= 1e-10 max(|oracle|, 1e-2 K);
derivatives: |gpu - oracle| <= 1e-6 max(|oracle|, 1e-3 K).

  * the 18 single options at paper scale (Section 5, Table 2 parameters), one option per
    launch of the batched entry point, and all 18 through the whole-GPU form;
  * the 32 costliest options of the 4096-option batch, priced inside the full batch in one
    launch (the launch the benchmark times);
  * 32 options through the adjoint at N = 1000: 16 of the 1024 puts inside the full
    1024-option launch, and 16 calls and bull spreads.
"""
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-10
GTOL = 1e-6
GOLD = os.path.join(os.path.dirname(__file__), "golden")
FIELDS = ("S0", "K", "K2", "sigma", "R", "T", "k", "N", "payoff")


def _ob():
    import paper_1110_2477_gb300 as ob
    return ob


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _table(recs):
    a = np.zeros(len(recs), W.OPTION_DTYPE)
    for i, r in enumerate(recs):
        for f in FIELDS:
            a[i][f] = r[f]
    return a


def _price(table, wide=False):
    import torch
    out, st = _ob().price(table, wide=wide)
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy()


def _assert_prices(table, out, st, ref, rst, what):
    assert np.array_equal(st, rst), (what, st.tolist(), rst.tolist())
    scale = np.maximum(np.abs(ref), 1e-2 * table["K"][:, None])
    err = np.abs(out - ref) / scale
    worst = int(np.argmax(err.max(axis=1)))
    assert err.max() <= RTOL, (what, worst, out[worst].tolist(), ref[worst].tolist(), table[worst])


def test_paper_scale_all_18_one_per_launch():
    g = _gold("paper_scale.json")
    t = _table(g["options"])
    assert np.array_equal(t, W.paper_scale())  # the stored records are the workload's
    ref, rst = np.array(g["ask_bid"]), np.array(g["status"], np.int32)
    out = np.zeros_like(ref)
    st = np.zeros(len(t), np.int32)
    for i in range(len(t)):
        o, s = _price(t[i:i + 1])
        out[i], st[i] = o[0], s[0]
    _assert_prices(t, out, st, ref, rst, "one option per launch")


def test_paper_scale_all_18_whole_gpu_form():
    g = _gold("paper_scale.json")
    t = _table(g["options"])
    ref, rst = np.array(g["ask_bid"]), np.array(g["status"], np.int32)
    out, st = _price(t, wide=True)
    _assert_prices(t, out, st, ref, rst, "whole-GPU form")


def test_batched_costliest_32_inside_full_batch():
    g = _gold("batched_costliest.json")
    full = W.batched_uneven()
    idx = np.array(g["index"])
    assert np.array_equal(full[idx], _table(g["options"]))
    out, st = _price(full)
    assert np.all(st == 0)
    ref, rst = np.array(g["ask_bid"]), np.array(g["status"], np.int32)
    _assert_prices(full[idx], out[idx], st[idx], ref, rst, "costliest of the batch")


def _greeks(table):
    import torch
    out, grad, st = _ob().greeks(table)
    torch.cuda.synchronize()
    return out.cpu().numpy(), grad.cpu().numpy(), st.cpu().numpy()


def _assert_greeks(table, out, grad, st, ref, rgrad, rst, what):
    _assert_prices(table, out, st, ref, rst, what)
    scale = np.maximum(np.abs(rgrad), 1e-3 * table["K"][:, None, None])
    err = np.abs(grad - rgrad) / scale
    worst = np.unravel_index(np.argmax(err), err.shape)
    assert err.max() <= GTOL, (what, worst, grad[worst[0]].tolist(), rgrad[worst[0]].tolist())


def test_greeks_sample_32():
    g = _gold("greeks_sample.json")
    t = _table(g["options"])
    ref, rgrad = np.array(g["ask_bid"]), np.array(g["grad"])
    rst = np.array(g["status"], np.int32)
    puts = W.greeks_puts()
    pidx = np.array(g["put_index"])
    npu = len(pidx)
    assert np.array_equal(t[:npu], puts[pidx])
    # the 16 puts inside the full 1024-option launch
    out, grad, st = _greeks(puts)
    _assert_greeks(t[:npu], out[pidx], grad[pidx], st[pidx], ref[:npu], rgrad[:npu], rst[:npu],
                   "puts inside the 1024-option launch")
    # the calls and spreads
    out, grad, st = _greeks(t[npu:])
    _assert_greeks(t[npu:], out, grad, st, ref[npu:], rgrad[npu:], rst[npu:], "calls and spreads")
