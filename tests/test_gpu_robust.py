"""Failure detection and concurrency of the C-ABI entry points, on the GPU.

  * The whole-GPU form's grid barrier waits are bounded: with a test control that keeps
    one CTA from ever arriving (read once per process, so the test runs in a child
    process), every option of that call reports OB_ERR_TIMEOUT with NaN prices, the context
    stays usable, and the next call prices normally.  No fault, trap or endless wait is
    involved: the other CTAs give up after a 200 ms limit and return.
  * Calls made concurrently on two streams, and from two host threads, are ordered by the
    library on the device and price as they do alone.
  * An allocation failure injected on the host (a pool size no GPU has) is reported as
    OB_ERR_NOMEM with nothing enqueued; the context stays usable.
"""
import json
import os
import subprocess
import sys
import threading

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RTOL = 1e-10

_WIDE_CHILD = r"""
import sys, json, numpy as np, torch
sys.path.insert(0, %(root)r)
import workloads as W, paper_1110_2477_gb300 as ob
t = W.concat(W.make(k=0.01, N=40), W.make(k=0.005, N=30, payoff=W.CALL),
             W.make(K=95.0, K2=105.0, k=0.01, N=20, payoff=W.SPREAD))
res = {}
for name, wide in (("first", True), ("second", True), ("batched", False)):
    out, st = ob.price(t, wide=wide)
    torch.cuda.synchronize()
    res[name] = {"out": out.cpu().numpy().tolist(), "st": st.cpu().numpy().tolist()}
print(json.dumps(res))
"""


def test_wide_barrier_timeout_reports_status_and_recovers():
    env = dict(os.environ, OB_WIDE_WAIT_MS="200", OB_TEST_WIDE_SKIP="1")
    r = subprocess.run([sys.executable, "-c", _WIDE_CHILD % {"root": ROOT}], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["first"]["st"] == [-4, -4, -4]
    assert np.all(np.isnan(np.array(res["first"]["out"])))
    assert res["second"]["st"] == [0, 0, 0] == res["batched"]["st"]
    a = np.array(res["second"]["out"])
    b = np.array(res["batched"]["out"])
    assert np.array_equal(a.view(np.int64), b.view(np.int64))


def _alone(table):
    import torch

    import paper_1110_2477_gb300 as ob
    out, st = ob.price(table)
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy()


def test_two_streams_price_as_alone():
    import torch

    import paper_1110_2477_gb300 as ob
    t1 = W.random_table(120, 7001, N_lo=20, N_hi=500)
    t2 = W.random_table(90, 7002, N_lo=20, N_hi=500)
    a1, s1 = _alone(t1)
    a2, s2 = _alone(t2)
    p1, p2 = ob.to_device(t1), ob.to_device(t2)
    c2 = ob.to_device(t2.copy())
    outs = []
    for rep in range(3):
        st1, st2 = torch.cuda.Stream(), torch.cuda.Stream()
        o1 = torch.empty((len(t1), 2), dtype=torch.float64, device="cuda")
        o2 = torch.empty((len(t2), 2), dtype=torch.float64, device="cuda")
        q1 = torch.empty(len(t1), dtype=torch.int32, device="cuda")
        q2 = torch.empty(len(t2), dtype=torch.int32, device="cuda")
        crr = torch.empty(len(t2), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        ob.ob_price_ask_bid(p1, len(t1), o1, q1, st1)
        ob.ob_price_ask_bid(p2, len(t2), o2, q2, st2)
        ob.ob_crr_american(c2, len(t2), crr, None, st1)
        torch.cuda.synchronize()
        outs.append((o1.cpu().numpy(), q1.cpu().numpy(), o2.cpu().numpy(), q2.cpu().numpy()))
    for o1, q1, o2, q2 in outs:
        assert np.array_equal(q1, s1) and np.array_equal(q2, s2)
        assert np.array_equal(o1.view(np.int64), a1.view(np.int64))
        assert np.array_equal(o2.view(np.int64), a2.view(np.int64))
    idx = np.array([0, 17, 55, 89])
    ref, rst = oracle.price_ask_bid(t2[idx], nthreads=4)
    scale = np.maximum(np.abs(ref), 1e-2 * t2["K"][idx][:, None])
    assert np.all(np.abs(outs[0][2][idx] - ref) <= RTOL * scale)


def test_two_host_threads_price_as_alone():
    import torch

    import paper_1110_2477_gb300 as ob
    tables = [W.random_table(60, 7100 + i, N_lo=20, N_hi=400) for i in range(2)]
    alone = [_alone(t) for t in tables]
    results = [None, None]
    errors = []

    def work(i):
        try:
            torch.cuda.set_device(0)
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                p = ob.to_device(tables[i])
                o = torch.empty((len(tables[i]), 2), dtype=torch.float64, device="cuda")
                q = torch.empty(len(tables[i]), dtype=torch.int32, device="cuda")
                for _ in range(3):
                    ob.ob_price_ask_bid(p, len(tables[i]), o, q, s)
                s.synchronize()
                results[i] = (o.cpu().numpy(), q.cpu().numpy())
        except Exception as e:  # reported below
            errors.append(repr(e))

    th = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join(timeout=300)
    assert not errors, errors
    for (o, q), (a, s) in zip(results, alone):
        assert np.array_equal(q, s)
        assert np.array_equal(o.view(np.int64), a.view(np.int64))


_NOMEM_CHILD = r"""
import sys, json, numpy as np, torch
sys.path.insert(0, %(root)r)
import workloads as W, paper_1110_2477_gb300 as ob
t = W.concat(W.make(k=0.01, N=40), W.make(k=0.005, N=30, payoff=W.CALL))
res = {}
for k in range(2):
    try:
        ob.price(t)
        torch.cuda.synchronize()
        res["price%d" % k] = "ok"
    except ob.ObError as e:
        res["price%d" % k] = str(e)
res["torch"] = float(torch.arange(10, device="cuda", dtype=torch.float64).sum().item())
print(json.dumps(res))
"""


def test_pool_allocation_failure_is_reported_and_the_context_stays_usable():
    """An allocation failure injected on the host side: a pool size no GPU has (OB_POOL_MB,
    read once per process, so the test runs in a child process).  cudaMalloc refuses it, the
    pooled call returns OB_ERR_NOMEM with nothing enqueued, a second call does the same, and
    the CUDA context stays usable."""
    env = dict(os.environ, OB_POOL_MB="1000000000")  # 1e9 MiB
    r = subprocess.run([sys.executable, "-c", _NOMEM_CHILD % {"root": ROOT}], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["price0"].endswith("(-6)"), res["price0"]
    assert res["price1"].endswith("(-6)"), res["price1"]
    assert res["torch"] == 45.0
