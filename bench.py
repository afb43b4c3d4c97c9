"""Benchmark: batched ask/bid pricing of 4096 uneven American options with
proportional transaction costs, FP64, one persistent launch per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is tree node updates per second
(ask and bid together; (N+1)(N+2)/2 updates per option), device-timed with
CUDA events on the launching stream, inputs resident in HBM.  `e2e` is the
same metric through the host-buffer C-ABI call (pinned host buffers, copies
inside the timed region).  `--impl reference` times the CPU oracle on the
host cores on a bounded sample of the same workload.

Under torchrun each rank prices its own batch of the same distribution
(weak scaling, no collective on the data path); the max over ranks of the
timed region sets the job time.

Other workloads (--workload): small (48 options, for profiler captures), crr
(65536 CRR puts at N = 2048 and one put at N = 20000), paper (18 paper-scale
single options, one per launch on the whole GPU), greeks (1024 puts, prices
and the 12 derivatives; --options n for a smaller case), path (the same puts,
the hedge along one random path each).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "tree node updates/s (ask+bid, FP64) batched; options/s with Greeks vs plain"
FP64_NOMINAL_TFLOPS = 1.25  # GB300 dense FP64: 152 SMs x 2.07 GHz x 2 DFMA lanes x 2 flops (context)
FLOPS_PER_MERGED_POINT = 10  # algorithmic FP64 flops per merged successor breakpoint: the low end
                             # of the c = 10-15 per (m_u + m_d) of the step-by-step count
CPU_SAMPLE = 48          # options of the batch the CPU oracle prices per step
# DRAM traffic of one k_tc_batched launch on the 4096-option batch, from an ncu capture
# recorded with the hash of the kernel's sources; reported only while the sources match
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "k_tc_batched_traffic.json")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1110_2477_gb300", "csrc", f)
                  for f in ("ob_tc.cuh", "ob_team.cuh", "ob_kern.cuh", "ob_batched16.cu",
                            "ob_batched_half.cu", "ob_lib.cu")]


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic():
    """DRAM bytes per launch of the batched kernel from the committed capture record, or None
    when the kernel's sources have changed since it was taken."""
    try:
        with open(TRAFFIC_RECORD) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("src_sha256") != kernel_source_hash():
        return None
    return int(rec["dram_read_bytes"]) + int(rec["dram_write_bytes"])


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def measure_fp64_peak(local):
    """FP64 FMA throughput of this GPU (ob_fp64_peak), with the clocks seen while it ran."""
    import paper_1110_2477_gb300 as ob
    sampler = ClockSampler(local)
    sampler.start()
    tf, ms = ob.ob_fp64_peak(1 << 17)
    clocks = sampler.stop()
    return {"tflops": tf, "ms": ms, "clocks": clocks,
            "how": "ob_fp64_peak: 8 CTAs x 256 threads per SM, 8 independent DFMA chains per thread, "
                   "CUDA events, fastest of 2 timed runs"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-greeks", action="store_true", help="skip the Greeks-vs-plain comparison")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the one-warp-per-option comparison kernel (for profiler captures)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default team width")
    ap.add_argument("--options", type=int, default=1024,
                    help="greeks and path workloads: the first n of the 1024 puts (smaller for profiling)")
    ap.add_argument("--workload", default="batched", choices=["batched", "small", "crr", "paper", "greeks", "path"],
                    help="batched: the 4096-option batch (the reported metric); small: 48 options "
                         "with N in [200, 600] (seed 321), for profiler captures")
    return ap.parse_args()


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    """The sum of x over the ranks (units that all ranks processed)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(table, seed=7):
    """The CPU oracle, as it stands, on a bounded random sample of the batch, all host cores."""
    import oracle
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(table), CPU_SAMPLE, replace=False)
    sample = table[idx]
    cores = os.cpu_count() or 1
    oracle.build()
    t0 = time.perf_counter()
    oracle.price_ask_bid(sample, nthreads=cores)
    dt = time.perf_counter() - t0
    nodes = int(np.sum(W.node_updates(sample)))
    return {"value": nodes / dt, "unit": "node updates/s", "cores": cores, "cpu_model": cpu_model(),
            "kind": "oracle",
            "sample": "%d random options of the 4096-option batch (seed %d), %d node updates, %.1f s"
                      % (CPU_SAMPLE, seed, nodes, dt)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    table = W.batched_uneven()
    oracle.build()
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(11)
    samples = [table[rng.choice(len(table), 16, replace=False)] for _ in range(args.warmup + args.steps)]
    for s in samples[:args.warmup]:
        oracle.price_ask_bid(s[:2], nthreads=cores)
    nodes = 0
    t0 = time.perf_counter()
    for s in samples[args.warmup:]:
        oracle.price_ask_bid(s, nthreads=cores)
        nodes += int(np.sum(W.node_updates(s)))
    dt = time.perf_counter() - t0
    v = nodes / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "node updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batched uneven 4096 (N~U{100..2000}, put/call/spread)",
                       "sample_per_step": "16 random options of the batch"},
            "cpu_baseline": {"value": v, "unit": "node updates/s", "cores": cores, "cpu_model": cpu_model(),
                             "kind": "oracle",
                             "sample": "16 random options per step of the 4096-option batch"},
            "e2e": {"value": v, "unit": "node updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_crr(args, rank, world, local):
    """The zero-cost limit at scale: 65536 CRR American puts, N = 2048 (seed 5), one
    ob_crr_american launch per step; then one put at N = 20000 (latency)."""
    import torch

    import paper_1110_2477_gb300 as ob
    dev = torch.device("cuda", local)
    peak = measure_fp64_peak(local)
    table = W.crr_puts() if rank == 0 else W.crr_puts(seed=5 + 1000 * rank)
    n = len(table)
    nodes = int(np.sum(table["N"].astype(np.int64) * (table["N"].astype(np.int64) + 1) // 2))
    params = ob.to_device(table, dev)
    out = torch.empty(n, dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        ob.ob_crr_american(params, n, out, st, stream)
    torch.cuda.synchronize(dev)
    assert int((st != 0).sum().item()) == 0
    sampler = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(world)
    sampler.start()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        ob.ob_crr_american(params, n, out, st, stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    job_s = max_over_ranks(sum(step_ms) / 1e3, world)
    value = world * nodes * args.steps / job_s
    # end to end: pinned host records in, prices out, copies inside the timed region
    pin_in = torch.from_numpy(table.view(np.uint8).reshape(-1).copy()).pin_memory()
    pin_out = torch.empty(n, dtype=torch.float64).pin_memory()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        params.copy_(pin_in, non_blocking=True)
        ob.ob_crr_american(params, n, out, st, stream)
        pin_out.copy_(out, non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    big = W.appendix_put(20000)
    bp = ob.to_device(big, dev)
    bo = torch.empty(1, dtype=torch.float64, device=dev)
    bw = torch.empty(1, dtype=torch.float64, device=dev)
    ob.ob_crr_american(bp, 1, bo, None, stream)
    ob.ob_crr_american_wide(bp, 1, bw, None, stream)
    a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    a.record(stream)
    ob.ob_crr_american(bp, 1, bo, None, stream)
    b.record(stream)
    ob.ob_crr_american_wide(bp, 1, bw, None, stream)
    c.record(stream)
    torch.cuda.synchronize(dev)
    if rank != 0:
        return
    avg = job_s / args.steps
    flops = 3.0 * nodes / avg / 1e12  # one DFMA (2 flops) and one DMUL per node
    line = {
        "metric": "CRR node updates/s (k=0, FP64)", "value": value, "unit": "node updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * avg,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "65536 CRR American puts, N=2048, batched-table distributions, k=0 "
                               "(seed 5)", "node_updates_per_step": nodes,
                   "l2": "flushed (256 MiB write) before every timed step"},
        "e2e": {"value": world * nodes * args.steps / e2e_s, "unit": "node updates/s",
                "h2d_bytes_per_step": int(table.nbytes), "d2h_bytes_per_step": int(n * 8)},
        "gpu_launches": args.steps,
        "roofline": {"bound": "alu", "achieved": flops, "peak": peak["tflops"], "unit": "TFLOP/s",
                     "frac": flops / peak["tflops"], "traffic": None,
                     "note": "3 FP64 flops per node (DFMA + DMUL) against the measured FP64 FMA peak "
                             "(ob_fp64_peak)", "peak_measurement": peak},
        "put_n20000": {"price": float(bo.item()), "one_warp_ms": a.elapsed_time(b),
                       "whole_gpu_price": float(bw.item()), "whole_gpu_ms": b.elapsed_time(c),
                       "paper_context": {"serial_ms": 638.26, "p8_ms": 114.3,
                                         "machine": "2 x Xeon E5405, 8 cores (Table 3)"}},
        "step_ms": step_ms, "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        sample = table[:: n // 64]
        t0 = time.perf_counter()
        oracle.crr_price(sample, nthreads=cores)
        dt = time.perf_counter() - t0
        sn = int(np.sum(sample["N"].astype(np.int64) * (sample["N"].astype(np.int64) + 1) // 2))
        line["cpu_baseline"] = {"value": sn / dt, "unit": "node updates/s", "cores": cores,
                                "kind": "oracle", "sample": "every %d-th option (%d options), %.2f s"
                                % (n // 64, len(sample), dt)}
    print(json.dumps(line), flush=True)


def run_paper(args, rank, world, local):
    """Paper-scale single options: put (K=100) and cash-settled bull spread (95/105),
    S0=100, sigma=0.2, R=0.1, T=0.25, k in {0.25%, 0.5%, 1%}, N in {1500, 3000, 6000};
    one option per launch on the whole GPU (ob_price_ask_bid_wide).  A step prices
    the 18 options in turn; each option is also timed once on one CTA."""
    import torch

    import paper_1110_2477_gb300 as ob
    dev = torch.device("cuda", local)
    table = W.paper_scale()
    n = len(table)
    nodes = W.node_updates(table)
    params = [ob.to_device(table[i:i + 1], dev) for i in range(n)]
    out = torch.empty((1, 2), dtype=torch.float64, device=dev)
    st = torch.empty(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        for i in range(n):
            ob.ob_price_ask_bid_wide(params[i], 1, out, st, stream)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
          for _ in range(args.steps)]
    prices = np.zeros((n, 2))
    barrier(world)
    sampler.start()
    for k in range(args.steps):
        for i in range(n):
            ev[k][i][0].record(stream)
            ob.ob_price_ask_bid_wide(params[i], 1, out, st, stream)
            ev[k][i][1].record(stream)
            if k == 0:
                prices[i] = out[0].cpu().numpy()
                assert int(st.item()) == 0
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = np.array([[a.elapsed_time(b) for a, b in row] for row in ev])
    job_s = max_over_ranks(ms.sum() / 1e3, world)
    value = world * float(nodes.sum()) * args.steps / job_s
    one_cta = []
    for i in range(n):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ob.ob_price_ask_bid(params[i], 1, out, st, stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        one_cta.append(a.elapsed_time(b))
    if rank != 0:
        return
    med = np.median(ms, axis=0)
    rows = [{"N": int(table["N"][i]), "payoff": ["put", "call", "spread"][int(table["payoff"][i])],
             "k": float(table["k"][i]), "ask": float(prices[i, 0]), "bid": float(prices[i, 1]),
             "wide_ms": round(float(med[i]), 2), "one_cta_ms": round(one_cta[i], 2)} for i in range(n)]
    line = {
        "metric": "paper-scale single options, one per launch on the whole GPU: node updates/s (ask+bid)",
        "value": value, "unit": "node updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * job_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "put K=100 and bull spread 95/105, S0=100, sigma=0.2, R=0.1, T=0.25, "
                               "k in {0.0025, 0.005, 0.01}, N in {1500, 3000, 6000}; 18 launches per step",
                   "node_updates_per_step": int(nodes.sum())},
        "gpu_launches": n * args.steps, "options": rows, "clocks": clocks,
        "paper_context": {"put_N1500_k0.005_serial_ms": 1983.7, "put_N1500_k0.005_8cores_ms": 376.8,
                          "spread_N1500_k0.01_serial_ms": 2005.2, "machine": "2 x Xeon E5405, 8 cores"},
    }
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        one = table[2:3]  # the N=1500 put at k=0.005
        t0 = time.perf_counter()
        oracle.price_ask_bid(one, nthreads=1)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": float(nodes[2]) / dt, "unit": "node updates/s", "cores": 1,
                                "kind": "oracle", "cpu_model": cpu_model(),
                                "sample": "the N=1500 put at k=0.005, one thread, %.2f s" % dt,
                                "alg1": alg1_speedups(one, dt, crr=False)}
        crr_one = W.appendix_put(20000)
        t0 = time.perf_counter()
        oracle.crr_price(crr_one)
        line["cpu_baseline"]["alg1_crr"] = alg1_speedups(crr_one, time.perf_counter() - t0, crr=True)
    print(json.dumps(line), flush=True)


def alg1_speedups(opt, serial_s, crr):
    """The paper's parallel scheme (Section 4.2, Algorithm 1) over the oracle's node steps on
    the host cores: time and speedup over the serial oracle for 1, 2, 4, 8, ... threads and
    blocks of L = 5 and 50 levels (the paper's Tables 2 and 3 shape)."""
    import oracle
    cores = os.cpu_count() or 1
    threads = sorted({p for p in (1, 2, 4, 8, 16, cores) if p <= cores})
    ref = oracle.crr_price(opt)[0] if crr else oracle.price_ask_bid(opt)[0][0]
    rows = []
    for p in threads:
        for L in (5, 50):
            t0 = time.perf_counter()
            out, st, _ = oracle.alg1_price(opt, p, L, crr=crr)
            dt = time.perf_counter() - t0
            rows.append({"threads": p, "L": L, "s": round(dt, 3), "speedup": round(serial_s / dt, 2),
                         "status": st, "bitwise_equal": bool(np.array_equal(out, ref))})
    return {"option": "N=%d %s, k=%g" % (int(opt["N"][0]), "CRR put" if crr else "put", float(opt["k"][0])),
            "serial_s": round(serial_s, 3), "cores": cores, "rows": rows}


def run_greeks(args, rank, world, local):
    """The adjoint workload: 1024 American puts, N = 1000 (seed 4), prices and the 12
    derivatives per option in one ob_greeks call per step; options/s against the plain
    pricing call on the same options."""
    import torch

    import paper_1110_2477_gb300 as ob
    dev = torch.device("cuda", local)
    table = W.greeks_puts()[:args.options]
    n = len(table)
    params = ob.to_device(table, dev)
    out = torch.empty((n, 2), dtype=torch.float64, device=dev)
    grad = torch.empty((n, 2, 6), dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        ob.ob_greeks(params, n, out, grad, st, stream)
    torch.cuda.synchronize(dev)
    assert int((st != 0).sum().item()) == 0
    sampler = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(world)
    sampler.start()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        ob.ob_greeks(params, n, out, grad, st, stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    job_s = max_over_ranks(sum(step_ms) / 1e3, world)
    pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ob.ob_price_ask_bid(params, n, out, st, stream)
    pa.record(stream)
    ob.ob_price_ask_bid(params, n, out, st, stream)
    pb.record(stream)
    torch.cuda.synchronize(dev)
    plain_s = pa.elapsed_time(pb) / 1e3
    u_points = ob.ob_get_stats()["u_points"]
    peak = measure_fp64_peak(local)
    if rank != 0:
        return
    value = world * n * args.steps / job_s
    # every level is evaluated once (the forward pass keeps the records of every level: each
    # option of this workload fits), counted as the pricing line counts it; the recording and
    # the reverse sweep's scatter are not counted
    g_flops = 1.0 * FLOPS_PER_MERGED_POINT * float(u_points)
    g_achieved = g_flops / (job_s / args.steps) / 1e12
    line = {
        "metric": "options/s with Greeks (ask, bid and 12 derivatives), FP64", "value": value,
        "unit": "options/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * job_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "%d American puts, N=1000, batched-table distributions (seed 4)" % n,
                   "node_updates_per_step": int(np.sum(W.node_updates(table))),
                   "l2": "flushed (256 MiB write) before every timed step"},
        "plain": {"value": n / plain_s, "unit": "options/s", "call": "ob_price_ask_bid"},
        "greeks_over_plain_time": (job_s / args.steps) / plain_s,
        "gpu_launches": 3 * args.steps, "step_ms": step_ms, "clocks": clocks,
        "roofline": {"bound": "alu", "achieved": g_achieved, "peak": peak["tflops"], "unit": "TFLOP/s",
                     "frac": g_achieved / peak["tflops"], "traffic": None,
                     "note": "algorithmic FP64 flops = 1 level evaluation (the forward pass, which "
                             "keeps the records of every level) x %d per merged successor breakpoint "
                             "(U of the pricing pass); recording and the reverse sweep are not "
                             "counted; peak = ob_fp64_peak" %
                             FLOPS_PER_MERGED_POINT, "peak_measurement": peak},
    }
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        sample = table[:cores]
        t0 = time.perf_counter()
        oracle.greeks(sample, nthreads=cores)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(sample) / dt, "unit": "options/s", "cores": cores,
                                "kind": "oracle", "sample": "the first %d options, forward-mode "
                                "dual numbers, %.1f s" % (len(sample), dt)}
    print(json.dumps(line), flush=True)


def run_path(args, rank, world, local):
    """The hedge along a path: the 1024 puts of the Greeks workload (N = 1000, seed 4), one
    random path per option (seed 8), prices plus both parties' holdings and cash at every node
    of the path and the buyer's stopping level in one ob_hedge_path call per step; options/s against
    the pricing call on the same options."""
    import torch

    import paper_1110_2477_gb300 as ob
    dev = torch.device("cuda", local)
    table = W.greeks_puts()[:args.options]
    n = len(table)
    S = int(table["N"].max())
    params = ob.to_device(table, dev)
    moves = torch.as_tensor(np.random.default_rng(8).integers(0, 2, (n, S)).astype(np.int8)).to(dev)
    out = torch.empty((n, 2), dtype=torch.float64, device=dev)
    hold = torch.empty((n, S + 1, 2), dtype=torch.float64, device=dev)
    cash = torch.empty_like(hold)
    stop = torch.empty(n, dtype=torch.int32, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        ob.ob_hedge_path(params, n, moves, S, out, hold, cash, stop, st, stream)
    torch.cuda.synchronize(dev)
    assert int((st != 0).sum().item()) == 0
    sampler = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(world)
    sampler.start()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        ob.ob_hedge_path(params, n, moves, S, out, hold, cash, stop, st, stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    job_s = max_over_ranks(sum(step_ms) / 1e3, world)
    pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ob.ob_price_ask_bid(params, n, out, st, stream)
    pa.record(stream)
    ob.ob_price_ask_bid(params, n, out, st, stream)
    pb.record(stream)
    torch.cuda.synchronize(dev)
    plain_s = pa.elapsed_time(pb) / 1e3
    u_points = ob.ob_get_stats()["u_points"]
    peak = measure_fp64_peak(local)
    if rank != 0:
        return
    value = world * n * args.steps / job_s
    p_flops = 1.0 * FLOPS_PER_MERGED_POINT * float(u_points)
    p_achieved = p_flops / (job_s / args.steps) / 1e12
    line = {
        "metric": "options/s with the hedge along a path (ask, bid, holdings, cash, stopping level), FP64",
        "value": value, "unit": "options/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * job_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "%d American puts, N=1000, batched-table distributions (seed 4), one "
                               "random path each (seed 8)" % n,
                   "node_updates_per_step": int(np.sum(W.node_updates(table))),
                   "l2": "flushed (256 MiB write) before every timed step"},
        "plain": {"value": n / plain_s, "unit": "options/s", "call": "ob_price_ask_bid"},
        "path_over_plain_time": (job_s / args.steps) / plain_s,
        "gpu_launches": (3 if n <= 8192 else 2) * args.steps, "step_ms": step_ms, "clocks": clocks,
        "roofline": {"bound": "alu", "achieved": p_achieved, "peak": peak["tflops"], "unit": "TFLOP/s",
                     "frac": p_achieved / peak["tflops"], "traffic": None,
                     "note": "algorithmic FP64 flops = %d per merged successor breakpoint of the "
                             "induction (U of the pricing pass, counted by the last pricing call); "
                             "the copies of the path's w and the rebalancing sweep are not counted; "
                             "peak = ob_fp64_peak" % FLOPS_PER_MERGED_POINT,
                     "peak_measurement": peak},
    }
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        sample = table[:cores]
        mv = moves[:cores].cpu().numpy()
        t0 = time.perf_counter()
        oracle.hedge_path(sample, mv, nthreads=cores)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(sample) / dt, "unit": "options/s", "cores": cores,
                                "kind": "oracle", "sample": "the first %d options and paths, %.1f s" %
                                (len(sample), dt)}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch

    import paper_1110_2477_gb300 as ob
    from paper_1110_2477_gb300 import _build
    _build.build()
    ob.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.workload == "crr":
        run_crr(args, rank, world, local)
        return
    if args.workload == "paper":
        run_paper(args, rank, world, local)
        return
    if args.workload == "path":
        run_path(args, rank, world, local)
        return
    if args.workload == "greeks":
        run_greeks(args, rank, world, local)
        return

    if args.workload == "small":
        table = W.random_table(48, 321 + rank, N_lo=200, N_hi=600)
    else:
        table = W.batched_uneven() if rank == 0 else W.random_table(4096, 3 + 1000 * rank)
    n = len(table)
    nodes_per_step = int(np.sum(W.node_updates(table)))
    params = ob.to_device(table, dev)
    out = torch.empty((n, 2), dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 126 MB of L2
    stream = torch.cuda.current_stream(dev)
    peak = measure_fp64_peak(local)

    # the autotuner picks the team width (CTA size, per-CTA breakpoint capacity) on a
    # sample of the batch, outside the timed region
    tuned = None
    if not args.no_autotune:
        tw, chip, tms = ob.ob_autotune(params, n, min(n, 1024), stream)
        tuned = {"team_warps": tw, "chip_points": chip, "half_teams": ob.ob_get_stats()["half_teams"],
                 "sample": min(n, 1024),
                 "sample_ms": {str(k): round(v, 2) for k, v in tms.items()}}
    for _ in range(args.warmup):
        ob.ob_price_ask_bid(params, n, out, st, stream)
    torch.cuda.synchronize(dev)
    assert int((st != 0).sum().item()) == 0, "options failed: %s" % st[st != 0][:8].tolist()
    stats = ob.ob_get_stats()

    sampler = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize(dev)
    sampler.start()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        ob.ob_price_ask_bid(params, n, out, st, stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    barrier(world)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(step_ms) / 1e3
    job_s = max_over_ranks(dev_s, world)
    job_nodes = sum_over_ranks(nodes_per_step, world)  # each rank prices its own batch
    value = job_nodes * args.steps / job_s

    # end to end through the host-buffer call: copies of inputs and results inside
    pin_in = torch.from_numpy(table.view(np.uint8).reshape(-1).copy()).pin_memory()
    pin_in_np = pin_in.numpy().view(W.OPTION_DTYPE)
    pin_out = torch.empty((n, 2), dtype=torch.float64).pin_memory()
    pin_st = torch.empty(n, dtype=torch.int32).pin_memory()
    ob.ob_price_ask_bid_host(pin_in_np, pin_out.numpy(), pin_st.numpy())
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ob.ob_price_ask_bid_host(pin_in_np, pin_out.numpy(), pin_st.numpy())
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": job_nodes * args.steps / e2e_s, "unit": "node updates/s",
           "h2d_bytes_per_step": int(table.nbytes),
           "d2h_bytes_per_step": int(pin_out.numel() * 8 + pin_st.numel() * 4)}

    # plain single-option kernel on the same batch (one warp per option, no queue)
    plain_s = None
    if not args.no_plain:
        ob.ob_price_ask_bid_plain(params, n, out, st, stream)
        torch.cuda.synchronize(dev)
        pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pa.record(stream)
        ob.ob_price_ask_bid_plain(params, n, out, st, stream)
        pb.record(stream)
        torch.cuda.synchronize(dev)
        plain_s = pa.elapsed_time(pb) / 1e3

    # options/s with Greeks vs plain pricing: 1024 puts, N = 1000 (seed 4)
    greeks_line = None
    if args.workload == "batched" and not args.no_greeks:
        gt = W.greeks_puts()
        gn = len(gt)
        gp = ob.to_device(gt, dev)
        gout = torch.empty((gn, 2), dtype=torch.float64, device=dev)
        ggrad = torch.empty((gn, 2, 6), dtype=torch.float64, device=dev)
        gst = torch.empty(gn, dtype=torch.int32, device=dev)
        ob.ob_greeks(gp, gn, gout, ggrad, gst, stream)
        ob.ob_price_ask_bid(gp, gn, gout, gst, stream)
        torch.cuda.synchronize(dev)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ob.ob_greeks(gp, gn, gout, ggrad, gst, stream)
        e1.record(stream)
        ob.ob_price_ask_bid(gp, gn, gout, gst, stream)
        e2.record(stream)
        torch.cuda.synchronize(dev)
        tg, tp = e0.elapsed_time(e1) / 1e3, e1.elapsed_time(e2) / 1e3
        assert int((gst != 0).sum().item()) == 0
        gnodes = int(np.sum(W.node_updates(gt)))
        greeks_line = {"workload": "1024 American puts, N=1000, batched-table distributions (seed 4)",
                       "greeks_options_per_s": gn / tg, "plain_options_per_s": gn / tp,
                       "greeks_node_updates_per_s": gnodes / tg, "greeks_over_plain_time": tg / tp}

    if rank != 0:
        return
    avg_step = dev_s / args.steps
    alg_flops = FLOPS_PER_MERGED_POINT * float(stats["u_points"])
    fma_flops = 2.0 * stats["u_points"] + 4.0 * stats["w_points"] + 2.0 * stats["z_points"]
    achieved = alg_flops / avg_step / 1e12
    traffic = recorded_traffic() if args.workload == "batched" else None
    line = {
        "metric": METRIC, "value": value, "unit": "node updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * job_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": ("batched uneven 4096: N~U{100..2000}, S0,K~U[80,120], sigma~U[0.1,0.5], "
                                "R~U[0,0.1], T~U[0.1,2], k~U[0,0.02], put/call/bull spread (width 10), seed 3")
                   if args.workload == "batched" else "small: 48 options, N in [200, 600], seed 321",
                   "options": n, "node_updates_per_step": nodes_per_step,
                   "l2": "flushed (256 MiB write) before every timed step",
                   "parallelism": "replicas (one batch per GPU)",
                   "team_warps": stats["team_warps"], "chip_points": stats["chip_points"],
                   "half_teams": stats["half_teams"],
                   "autotune": tuned,
                   "launch": "CUDA graph replay" if stats["graph"] == 2 else
                             ("CUDA graph" if stats["graph"] == 1 else "direct")},
        "options_per_s": world * n * args.steps / job_s,
        "plain": None if plain_s is None else {
            "value": nodes_per_step / plain_s, "unit": "node updates/s", "options_per_s": n / plain_s,
            "kernel": "one warp per option, index order"},
        "e2e": e2e,
        "gpu_launches": 4 * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak["tflops"],
                     "unit": "TFLOP/s", "frac": achieved / peak["tflops"], "traffic": traffic,
                     "note": "algorithmic FP64 flops = %d per merged successor breakpoint (U per step, "
                             "counted by the kernel); peak = measured FP64 FMA throughput of this GPU "
                             "(ob_fp64_peak); traffic = DRAM bytes read + written by one k_tc_batched "
                             "launch of this workload from the committed ncu record (null when the "
                             "kernel's sources changed since)" % FLOPS_PER_MERGED_POINT,
                     "fma_count": {"flops_per_step": fma_flops, "tflops": fma_flops / avg_step / 1e12,
                                   "frac": fma_flops / avg_step / 1e12 / peak["tflops"],
                                   "what": "2U + 4W + 2Z: the FMAs the kernel issues per merged point, "
                                           "point of w and point of z"},
                     "peak_measurement": peak},
        "breakpoints": {"u_points": stats["u_points"], "w_points": stats["w_points"],
                        "z_points": stats["z_points"], "max_level_points": stats["max_level_points"],
                        "retried": stats["retried"]},
        "step_ms": step_ms, "wall_s": wall, "clocks": clocks,
    }
    if greeks_line is not None:
        line["greeks"] = greeks_line
    if not args.no_cpu_baseline and world >= 1:
        line["cpu_baseline"] = cpu_baseline(table)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
