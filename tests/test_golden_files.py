"""The stored oracle values of the full-size parity cases (tests/golden/*.json, written by
tests/golden/make_golden.py) describe the workloads' own records and are reproduced by the
oracle as it stands (checked on the cheaper stored options; the oracle is deterministic,
so the values must agree to the bit)."""
import json
import os

import numpy as np

import oracle
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
FIELDS = ("S0", "K", "K2", "sigma", "R", "T", "k", "N", "payoff")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _table(recs):
    a = np.zeros(len(recs), W.OPTION_DTYPE)
    for i, r in enumerate(recs):
        for f in FIELDS:
            a[i][f] = r[f]
    return a


def test_stored_records_are_the_workloads():
    g = _gold("paper_scale.json")
    assert np.array_equal(_table(g["options"]), W.paper_scale())
    g = _gold("batched_costliest.json")
    full = W.batched_uneven()
    assert len(g["index"]) == 32 == len(set(g["index"]))
    assert np.array_equal(_table(g["options"]), full[np.array(g["index"])])
    g = _gold("greeks_sample.json")
    t = _table(g["options"])
    assert len(t) == 32
    assert np.array_equal(t[:16], W.greeks_puts()[np.array(g["put_index"])])
    assert set(t["payoff"][16:].tolist()) <= {W.CALL, W.SPREAD} and np.all(t["N"] == 1000)
    for name in ("paper_scale.json", "batched_costliest.json", "greeks_sample.json"):
        g = _gold(name)
        assert all(s == 0 for s in g["status"]), name
        assert np.all(np.isfinite(np.array(g["ask_bid"]))), name


def test_stored_values_reproduce():
    g = _gold("paper_scale.json")
    t = _table(g["options"])
    out, st = oracle.price_ask_bid(t[:1])  # the N = 1500 put at k = 0.25 %
    assert st[0] == 0 and np.array_equal(out[0], np.array(g["ask_bid"][0]))
    g = _gold("greeks_sample.json")
    t = _table(g["options"])
    out, grad, st = oracle.greeks(t[:2], nthreads=2)
    assert np.array_equal(out, np.array(g["ask_bid"][:2]))
    assert np.array_equal(grad, np.array(g["grad"][:2]))
