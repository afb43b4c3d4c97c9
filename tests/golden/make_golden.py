"""Write the stored oracle values of the full-size parity cases.

Run from the repository root:  python tests/golden/make_golden.py [paper|batched|greeks|all]

Every value written here comes from ``oracle/`` (the plain FP64 CPU
implementation) and nothing else; the option records come from the seeded
generators in ``workloads``.  The GPU tests compare the CUDA path with these
files element by element (prices at 1e-10 relative with a 1e-2 K floor,
derivatives at 1e-6 relative with a 1e-3 K floor).

Files:
  paper_scale.json        the 18 single options at paper scale (Section 5, the
                          parameters of Table 2: put K = 100 and cash-settled bull
                          spread 95/105, S0 = 100, sigma = 0.2, R = 0.1, T = 0.25,
                          k in {0.25 %, 0.5 %, 1 %}, N in {1500, 3000, 6000})
  batched_costliest.json  the 32 costliest options of the 4096-option batch (seed 3):
                          24 by predicted work (node updates x predicted breakpoints
                          per node) and the 8 calls / spreads with the largest
                          k / (sigma sqrt(T/N)) not already taken -- the options whose
                          nodes hold thousands of breakpoints
  greeks_sample.json      32 options through the derivative path at N = 1000: 16 of the
                          1024 puts (seed 4, every 64th) and 16 calls and bull spreads
                          drawn from the same distributions (seed 44)

Selecting which options to store uses the same breakpoint-count model as the
library's queue ordering, restated here; it picks cases and computes no
expected value.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

FIELDS = ("S0", "K", "K2", "sigma", "R", "T", "k", "N", "payoff")


def predicted_work(t):
    """Node updates times predicted breakpoints per node (both parties)."""
    N = t["N"].astype(np.float64)
    sd = t["sigma"] * np.sqrt(t["T"] / N)
    x = np.where(t["k"] > 0, t["k"] / sd, 0.0)
    m = np.full(len(t), 2.0)
    big = x > 1.0
    call, spread = t["payoff"] == W.CALL, t["payoff"] == W.SPREAD
    m[call & big] += 1.5 * x[call & big]
    m[spread & big] += x[spread & big] ** 2
    return (N + 1) * (N + 2) / 2 * m, x


def records(t):
    return [{f: (int(r[f]) if f in ("N", "payoff") else float(r[f])) for f in FIELDS} for r in t]


def table_of(recs):
    a = np.zeros(len(recs), W.OPTION_DTYPE)
    for i, r in enumerate(recs):
        for f in FIELDS:
            a[i][f] = r[f]
    return a


def price_in_cost_order(t):
    """Oracle prices, heaviest option first on the thread pool."""
    cost, _ = predicted_work(t)
    order = np.argsort(-cost, kind="stable")
    t0 = time.perf_counter()
    out, st = oracle.price_ask_bid(t[order], nthreads=os.cpu_count() or 1)
    res = np.empty_like(out)
    rst = np.empty_like(st)
    res[order] = out
    rst[order] = st
    return res, rst, time.perf_counter() - t0


def write(name, payload):
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        json.dump(payload, f, indent=1)
    print("wrote", path, flush=True)


def make_paper():
    t = W.paper_scale()
    out, st, dt = price_in_cost_order(t)
    write("paper_scale.json", {
        "citation": "Zhang, Roux, Zastawniak (2011), Section 5 and Table 2: American put K = 100 and "
                    "cash-settled bull spread 95/105, S0 = 100, sigma = 0.2, R = 0.1, T = 0.25; "
                    "k in {0.0025, 0.005, 0.01}, N in {1500, 3000, 6000}",
        "generator": "tests/golden/make_golden.py paper (oracle.price_ask_bid, FP64, CPU)",
        "oracle_seconds": round(dt, 1),
        "options": records(t), "ask_bid": out.tolist(), "status": st.tolist()})


def make_batched():
    t = W.batched_uneven()
    cost, x = predicted_work(t)
    by_cost = list(np.argsort(-cost, kind="stable")[:24])
    heavy = np.where(t["payoff"] != W.PUT)[0]
    by_x = [int(i) for i in heavy[np.argsort(-x[heavy], kind="stable")] if i not in by_cost][:8]
    idx = np.array(sorted(int(i) for i in by_cost + by_x))
    out, st, dt = price_in_cost_order(t[idx])
    write("batched_costliest.json", {
        "citation": "Batched uneven workload (4096 options, seed 3): N ~ U{100..2000}, S0, K ~ U[80,120], "
                    "sigma ~ U[0.1,0.5], R ~ U[0,0.1], T ~ U[0.1,2], k ~ U[0,0.02], put / call / "
                    "bull spread (width 10); the induction of Section 3 (Algorithms 3.1, 3.5)",
        "generator": "tests/golden/make_golden.py batched (oracle.price_ask_bid, FP64, CPU)",
        "selection": "24 largest predicted work, then 8 calls/spreads with the largest k/(sigma sqrt(T/N))",
        "oracle_seconds": round(dt, 1),
        "index": idx.tolist(), "options": records(t[idx]), "ask_bid": out.tolist(),
        "status": st.tolist()})


def make_greeks():
    puts = W.greeks_puts()
    pidx = np.arange(0, len(puts), 64)
    other = W.random_table(16, 44, payoffs=(W.CALL, W.SPREAD), fixed_N=1000)
    t = W.concat(puts[pidx], other)
    cost, _ = predicted_work(t)
    order = np.argsort(-cost, kind="stable")
    t0 = time.perf_counter()
    out, grad, st = oracle.greeks(t[order], nthreads=os.cpu_count() or 1)
    dt = time.perf_counter() - t0
    r_out, r_grad, r_st = np.empty_like(out), np.empty_like(grad), np.empty_like(st)
    r_out[order], r_grad[order], r_st[order] = out, grad, st
    write("greeks_sample.json", {
        "citation": "Derivatives of ask and bid (Section 3 induction) with respect to (S0, K, sigma, R, T, k) "
                    "by forward-mode dual numbers; 16 of the 1024 N = 1000 puts (seed 4, every 64th) and "
                    "16 calls / bull spreads at N = 1000 from the same distributions (seed 44)",
        "generator": "tests/golden/make_golden.py greeks (oracle.greeks, FP64, CPU)",
        "oracle_seconds": round(dt, 1),
        "put_index": pidx.tolist(), "options": records(t), "ask_bid": r_out.tolist(),
        "grad": r_grad.tolist(), "status": r_st.tolist()})


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "all"
    oracle.build()
    if which in ("paper", "all"):
        make_paper()
    if which in ("batched", "all"):
        make_batched()
    if which in ("greeks", "all"):
        make_greeks()
