"""Benchmark of the B300 radial-pattern keyword search (one JSON line on stdout).

Workload (N = 1): the medium synthetic knowledge graph - R-MAT
(a=.57, b=.19, c=.19), 2^21 nodes, 2^25 sampled edges, int32 CSR both
directions - with 64 queries issued one at a time (|C| in 2..4, |M| in 0..4,
keyword ranks 100..20,000, k = 20, max depth 8).  One step = the 64 queries.

  value      queries/s with the query keyword ids already in device memory and
             results left there (rpq_search_device, CUDA graph per shape),
             CUDA events on the library's stream, L2 flushed between steps
  e2e        the same through rpq_search (host buffers in and out, one
             synchronous call per query), wall clock
  roofline   the expansion kernel: algorithmic bytes / its device time,
             measured with CUDA events around each launch (profiling pass)
  cpu_baseline  the serial CPU oracle on a bounded sample of the workload

``--impl reference`` times the CPU oracle itself as the reference arm.
Multi-GPU (torchrun): queries are independent, every rank runs its own copy
of the workload on its GPU (replicas, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RPQ queries/sec and GTEPS (batched vs one-at-a-time, bit-exact); p50/p99 latency"
WORKLOAD = ("medium: R-MAT(.57,.19,.19) 2^21 nodes, 2^25 sampled edges, symmetric int32 CSR; "
            "64 RPQs one at a time, |C| 2-4, |M| 0-4, ranks 100-20000, k=20, L=8")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6400.0
# DRAM bytes per expansion launch from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the kernel source with this SHA-1 prefix; the
# value is reported only while the kernel source is unchanged.
NCU_TRAFFIC = {"sha1": "9e025e4dbd13", "bytes_per_launch": 5063236}


def expand_source_sha() -> str:
    """SHA-1 prefix of the expansion section of search_kernels.cu (k_expand and
    its helpers): the stored DRAM traffic is reported only while it is unchanged."""
    text = open(os.path.join(ROOT, "paper_2001_06770_b300", "csrc", "search_kernels.cu")).read()
    a = text.index("// ----------------------------------------------------------- level: expand")
    b = text.index("// ------------------------------------------------------ persistent run kernel")
    return hashlib.sha1(text[a:b].encode()).hexdigest()[:12]


def hbm_peak():
    try:
        pk = json.load(open(PEAKS_FILE))
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the raw samples (RPQ_CLOCKS_DIR, else the temporary directory); the
        # JSON line carries their summary
        out = os.environ.get("RPQ_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 6:
                continue
            try:
                sm.append(float(p[0]))
                mx = max(mx, float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[2:6]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_cpu() -> dict:
    """Host cores and CPU model (the oracle and RAKS-CPU run there)."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "model": model}


def oracle_sample(ds, qs, n, act=None, budget_s=20.0):
    """Serial oracle on the first n queries, stopping early once budget_s
    seconds are spent (at least one query): (queries/s, seconds, queries)."""
    import oracle
    if n <= 0:
        return None, 0.0, 0
    if act is None:
        act = oracle.dataset_activation(ds)
    t = time.perf_counter()
    done = 0
    for q in qs[:n]:
        oracle.search(ds, act.a, q.central, q.marginal, q.k, q.max_depth, q.gamma)
        done += 1
        if time.perf_counter() - t >= budget_s:
            break
    dt = time.perf_counter() - t
    return done / dt, dt, done


def _oracle_worker(args):
    """One process of the query-parallel oracle: its share of the queries,
    timed after the dataset and activation levels are ready."""
    ds_name, qs, budget_s = args
    sys.path.insert(0, ROOT)
    import oracle
    import rpqgen
    ds = rpqgen.make_dataset(ds_name)
    act = oracle.dataset_activation(ds)
    t = time.perf_counter()
    done = 0
    for q in qs:
        oracle.search(ds, act.a, q.central, q.marginal, q.k, q.max_depth, q.gamma)
        done += 1
        if time.perf_counter() - t >= budget_s:
            break
    return done, time.perf_counter() - t


def oracle_parallel_sample(ds_name, qs, per_core=2, budget_s=20.0):
    """The oracle query-parallel over all host cores, one process per core
    (spawned, so no CUDA state is inherited): (queries/s, processes, queries)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    shares = [(ds_name, qs[i::cores][:per_core], budget_s) for i in range(cores)]
    shares = [sh for sh in shares if sh[1]]
    with mp.get_context("spawn").Pool(len(shares)) as pool:
        out = pool.map(_oracle_worker, shares)
    done = sum(d for d, _ in out)
    return done / max(t for _, t in out), len(shares), done


def raks_cpu_sample(ds, qs, n, budget_s=20.0):
    """The paper's multi-core CPU search (OpenMP, all host cores) on the first
    n queries, stopping early after budget_s seconds: (queries/s, seconds,
    queries, threads)."""
    import raks_cpu
    a = raks_cpu.activation(ds)
    t = time.perf_counter()
    done = 0
    for q in qs[:n]:
        raks_cpu.search(ds, a, q.central, q.marginal, q.k, q.max_depth, q.gamma)
        done += 1
        if time.perf_counter() - t >= budget_s:
            break
    dt = time.perf_counter() - t
    return done / dt, dt, done, raks_cpu.threads()


def run_reference(args):
    ws, rank, _ = dist_init()
    if rank != 0:
        return 0
    import oracle
    import rpqgen
    wl = WORKLOADS[args.workload]
    ds = rpqgen.make_dataset(wl["ds"])
    qs = rpqgen.workload_queries(wl["queries"], ds)
    act = oracle.dataset_activation(ds)
    times = []
    for s in range(args.warmup + args.steps):
        q = qs[s % len(qs)]
        t = time.perf_counter()
        oracle.search(ds, act.a, q.central, q.marginal, q.k, q.max_depth, q.gamma)
        if s >= args.warmup:
            times.append(time.perf_counter() - t)
    total = sum(times)
    qps = args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": wl["desc"], "step": "one query of the workload (cycling)"},
            "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} queries of the {len(qs)}, serial C oracle, one core"},
            "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


WORKLOADS = {
    "medium": dict(ds="medium", queries="medium", mode="single", desc=WORKLOAD),
    "tiny": dict(ds="tiny", queries="tiny", mode="single",
                 desc="tiny: R-MAT 2^14 nodes, one RPQ (smoke and multi-process checks, not a bench line)"),
    "large": dict(ds="large", queries="large", mode="single",
                  desc="large: Chung-Lu (exponent 2.1) 5e7 nodes, 4e8 sampled edges, symmetric int32 CSR; "
                       "256 RPQs one at a time, |C| = |M| = 3, ranks 100-20000, k=20, L=8"),
    "batched": dict(ds="large", queries="batched", mode="batch",
                    desc="batched: large graph; 4096 RPQs of uneven shape (|C| 2-6, |M| 0-8, head/tail keywords, "
                         "k in {5,10,20}, L=8) in one rpq_search_batch call"),
    "served": dict(ds="medium", queries="served", mode="serve",
                   desc="served: medium graph; 20000 RPQs (shapes as batched) arriving as a Poisson stream, "
                        "continuous batching under a 16 GB slot budget"),
}


def expand_roofline(kg, qs, stats, workload="medium"):
    """Profiling pass: device time of each kernel class, and the expansion
    kernel's algorithmic bytes per second against the measured HBM peak.  The
    stored ncu DRAM traffic applies to the medium workload's 64 queries only."""
    kg.set_profiling(True)
    for q in qs:
        kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
    prof = kg.profile(reset=True)
    kg.set_profiling(False)
    exp_ms, exp_launches = prof["expand"]
    units = sum(s["work_units"] for s in stats)
    items = sum(s["work_items"] for s in stats)
    hits = sum(s["hits_central"] + s["hits_marginal"] for s in stats)
    # activations the expansion kernel executed (E_act less the skipped final marginal levels)
    e_act = sum(s["e_act_central"] + s["e_act_marginal"] - s["e_act_skipped"] for s in stats)
    alg_bytes = 4 * units + e_act + 2 * hits + 10 * items      # adjacency, level checks, writes, items
    achieved = alg_bytes / (exp_ms / 1e3) / 1e9 if exp_ms > 0 else 0.0
    peak, peak_kind = hbm_peak()
    traffic = (NCU_TRAFFIC["bytes_per_launch"]
               if workload == "medium" and len(qs) == 64 and NCU_TRAFFIC["sha1"] == expand_source_sha() else None)
    total_ms = sum(v[0] for v in prof.values())
    avg_s = exp_ms / 1e3 / max(exp_launches, 1)
    dram_gbs = traffic / avg_s / 1e9 if traffic and avg_s > 0 else None
    roof = {"bound": "hbm", "kernel": "k_expand", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
            "dram_gbs": dram_gbs, "dram_frac": dram_gbs / peak if dram_gbs else None,
            "alg_bytes_per_launch": alg_bytes / max(exp_launches, 1),
            "avg_launch_us": 1e3 * exp_ms / max(exp_launches, 1), "launches": exp_launches,
            "share_of_device_time": exp_ms / total_ms if total_ms else None}
    return roof, {k: v[0] for k, v in prof.items()}


def base_line(args, ws, wl, value, t_step, steps):
    return {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": ws, "steps": steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic", "tuning": args.tuning}


def run(args):
    ws, rank, local = dist_init()
    import torch
    import paper_2001_06770_b300 as rpq
    import rpqgen

    wl = WORKLOADS[args.workload]
    torch.cuda.set_device(local)
    ds = rpqgen.make_dataset(wl["ds"])
    qs = rpqgen.workload_queries(wl["queries"], ds)
    if args.queries:
        qs = qs[:args.queries]
    kg = rpq.KG.from_dataset(ds)
    # work-split parameters picked by the library's autotuner on a sample
    tuned = kg.autotune(qs[:args.tune_queries], repeats=2) if args.autotune else kg.tuning()
    args.tuning = tuned
    if wl["mode"] == "batch":
        line = run_batch(args, ws, rank, local, wl, ds, qs, kg)
    elif wl["mode"] == "serve":
        line = run_serve(args, ws, rank, local, wl, ds, qs, kg)
    else:
        line = run_single(args, ws, rank, local, wl, ds, qs, kg)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    kg.close()
    return 0


def run_single(args, ws, rank, local, wl, ds, qs, kg):
    import torch
    import paper_2001_06770_b300 as rpq
    nq = len(qs)
    stream = torch.cuda.ExternalStream(kg.slot_stream(0))
    # device-resident inputs and outputs
    kw_dev = [torch.tensor(list(q.central) + list(q.marginal), dtype=torch.int32, device="cuda") for q in qs]
    out_dev = torch.zeros((nq, 64 * 24), dtype=torch.uint8, device="cuda")
    nout_dev = torch.zeros(nq, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # 256 MB > 126 MB L2
    torch.cuda.synchronize()

    def step_device():
        for i, q in enumerate(qs):
            kg.search_device(kw_dev[i].data_ptr(), len(q.central), len(q.marginal), q.k, q.max_depth, q.gamma,
                             out_dev[i].data_ptr(), nout_dev[i:].data_ptr())

    # per-query statistics (E_act etc.) and correctness of the device path
    stats, host_res = [], []
    for q in qs:
        r, st = kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
        stats.append(st)
        host_res.append(r)
    e_act = sum(s["e_act_central"] + s["e_act_marginal"] for s in stats)
    launches_per_step = sum(st["kernels"] for st in stats)

    for _ in range(args.warmup):
        step_device()
    kg.sync_device()
    for i in range(nq):   # device path returns the host path's results
        got = np.frombuffer(out_dev[i].cpu().numpy().tobytes()[:24 * int(nout_dev[i].item())], rpq.RESULT_DTYPE)
        assert got.tobytes() == host_res[i].tobytes(), f"device/host mismatch on query {i}"

    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    step_ms = []
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.zero_()                       # L2 flush, outside the timed events
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step_device()
            b.record(stream)
            b.synchronize()
            step_ms.append(a.elapsed_time(b))
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    kg.sync_device()
    t_dev = allmax(ws, sum(step_ms) / 1e3)
    value = ws * nq * args.steps / t_dev

    # end to end through the host API: keyword ids in, results out, per call
    lat = []
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for q in qs:
            t = time.perf_counter()
            kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
            lat.append(time.perf_counter() - t)
    t_e2e = allmax(ws, time.perf_counter() - t0)
    e2e = ws * nq * args.steps / t_e2e
    h2d = 88 * nq                                  # parameter block with the keyword ids, per query
    d2h = sum(24 * q.k + 600 for q in qs)          # results + control block (600 B), per query

    # batched: all queries in one rpq_search_batch call (concurrent slots)
    kg.search_batch(qs)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        kg.search_batch(qs)
    t_b = allmax(ws, time.perf_counter() - t0)
    batched = ws * nq * args.steps / t_b

    roof, kms = expand_roofline(kg, qs, stats, args.workload)
    if rank != 0:
        return None
    cpu_qps, cpu_s, cpu_n = oracle_sample(ds, qs, args.cpu_sample)
    mc = raks_cpu_sample(ds, qs, args.cpu_sample * 2) if args.cpu_sample else None
    # query-parallel oracle on every host core (one process each) where a
    # process's copy of the graph is small enough (not on the 50M-node graph)
    par = oracle_parallel_sample(wl["ds"], qs) if args.cpu_sample and kg.n <= (1 << 22) else None
    line = base_line(args, ws, wl, value, t_dev / args.steps, args.steps)
    line.update({
        "config": {"workload": wl["desc"], "queries_per_step": nq, "n": kg.n, "m2": kg.m2, "abar": ds.abar,
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{ws}"},
        "gteps": e_act * ws * args.steps / t_dev / 1e9,
        "e_act_per_step": e_act,
        "e_act_skipped_per_step": sum(s["e_act_skipped"] for s in stats),
        "batched_qps": batched,
        "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99))},
        "e2e": {"value": e2e, "unit": "queries/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roof,
        "kernel_ms_per_step": kms,
        "cpu_baseline": ({"value": par[0], "unit": "queries/s", "cores": par[1], "kind": "oracle",
                          "sample": f"{par[2]} of the {nq} queries dealt round-robin to {par[1]} oracle "
                                    f"processes (one per core), throughput over the slowest process"}
                         if par else
                         {"value": cpu_qps, "unit": "queries/s", "cores": 1, "kind": "oracle",
                          "sample": f"first {cpu_n} of the {nq} queries, serial C oracle, {cpu_s:.1f} s"}),
        "host_cpu": host_cpu(),
        "cpu_baseline_one_core": {"value": cpu_qps, "unit": "queries/s", "cores": 1, "kind": "oracle",
                                  "sample": f"first {cpu_n} of the {nq} queries, serial C oracle, {cpu_s:.1f} s"},
        "raks_cpu": None if mc is None else {
            "value": mc[0], "unit": "queries/s", "threads": mc[3], "kind": "paper's multi-core CPU search (OpenMP)",
            "sample": f"first {mc[2]} of the {nq} queries, {mc[1]:.1f} s"},
        "clocks": clk,
    })
    return line


def run_batch(args, ws, rank, local, wl, ds, qs, kg):
    """All queries in one rpq_search_batch call per step; a sample is also run
    one at a time and must give identical results."""
    nq = len(qs)
    res0 = kg.search_batch(qs)
    assert all(st == 0 for _, _, st in res0), "batch query failed"
    sample = list(range(0, nq, max(1, nq // 128)))
    t0 = time.perf_counter()
    for i in sample:
        r, _ = kg.search(qs[i].central, qs[i].marginal, qs[i].k, qs[i].max_depth, qs[i].gamma)
        assert r.tobytes() == res0[i][0].tobytes(), f"batched result differs from one-at-a-time on query {i}"
    one_qps = len(sample) / (time.perf_counter() - t0)
    for _ in range(max(0, args.warmup - 1)):
        kg.search_batch(qs)
    clocks = Clocks(local)
    barrier(ws)
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        out = kg.search_batch(qs)
    t = allmax(ws, time.perf_counter() - t0)
    clk = clocks.stop()
    value = ws * nq * args.steps / t
    stats = [st for _, st, _ in out]
    e_act = sum(s["e_act_central"] + s["e_act_marginal"] for s in stats)
    sstats = [stats[i] for i in sample]
    roof, kms = expand_roofline(kg, [qs[i] for i in sample], sstats, args.workload)
    if rank != 0:
        return None
    cpu_qps, cpu_s, cpu_n = oracle_sample(ds, qs, args.cpu_sample)
    line = base_line(args, ws, wl, value, t / args.steps, args.steps)
    line.update({
        "config": {"workload": wl["desc"], "queries_per_step": nq, "n": kg.n, "m2": kg.m2, "abar": ds.abar,
                   "slots": kg.tuning()["batch_slots"], "l2": "inputs larger than L2 (3 GB adjacency)", "parallelism": f"replicas x{ws}"},
        "gteps": e_act * ws * args.steps / t / 1e9,
        "one_at_a_time_qps": one_qps,
        "batched_vs_one_at_a_time": value / (ws * one_qps),
        "equal_results_checked": len(sample),
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 88 * nq,
                "d2h_bytes_per_step": sum(24 * q.k + 600 for q in qs)},
        "gpu_launches": sum(s["kernels"] for s in stats) * args.steps,
        "roofline": roof, "kernel_ms_per_step_sample": kms,
        "cpu_baseline": {"value": cpu_qps, "unit": "queries/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {cpu_n} of the {nq} queries, serial C oracle, {cpu_s:.1f} s"},
        "clocks": clk,
    })
    return line


def run_serve(args, ws, rank, local, wl, ds, qs, kg):
    """Poisson arrival streams at several rates, served with continuous
    batching under a 16 GB slot budget; each result must equal the query run
    alone."""
    import paper_2001_06770_b300 as rpq
    import rpqgen
    nq = len(qs)
    srv = rpq.Server(kg, budget_bytes=16 << 30, max_slots=256)
    info = srv.info()
    sample = list(range(0, nq, max(1, nq // 64)))
    alone = {i: kg.search(qs[i].central, qs[i].marginal, qs[i].k, qs[i].max_depth, qs[i].gamma)[0] for i in sample}
    t0 = time.perf_counter()
    for i in sample:
        kg.search(qs[i].central, qs[i].marginal, qs[i].k, qs[i].max_depth, qs[i].gamma)
    one_qps = len(sample) / (time.perf_counter() - t0)
    srv.replay(qs[:2000], np.zeros(2000))                 # warm-up: graphs of every slot
    rates = [5000.0, 10000.0, 20000.0, 50000.0]
    per_rate = []
    clocks = Clocks(local)
    clocks.start()
    def serve_at(rate, below=False):
        arr = rpqgen.poisson_arrivals(nq, rate, seed=7)
        res, lat, status, wall = srv.replay(qs, arr)
        assert (status == 0).all()
        for i in sample:
            assert res[i].tobytes() == alone[i].tobytes(), f"served result differs from alone on query {i}"
        per_rate.append({"rate_per_s": rate, "qps": nq / wall, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                         "p99_ms": 1e3 * float(np.percentile(lat, 99)), "wall_s": wall,
                         "below_capacity": below})

    for rate in rates:
        serve_at(rate)
    # the configured rates can exceed the server's capacity (then latency is
    # queueing); two more streams below the measured capacity show service latency
    cap = max(r["qps"] for r in per_rate)
    for f in (0.5, 0.8):
        serve_at(round(f * cap), below=True)
    clk = clocks.stop()
    srv.close()
    if rank != 0:
        return None
    best = max((r for r in per_rate if not r["below_capacity"]), key=lambda r: r["qps"])
    cpu_qps, cpu_s, cpu_n = oracle_sample(ds, qs, args.cpu_sample)
    line = base_line(args, ws, wl, ws * best["qps"], best["wall_s"], 1)
    line.update({
        "config": {"workload": wl["desc"], "queries": nq, "n": kg.n, "m2": kg.m2, "slots": info["slots"],
                   "slot_bytes": info["slot_bytes"], "budget_bytes": 16 << 30, "l2": "inputs larger than L2",
                   "parallelism": f"replicas x{ws}"},
        "per_rate": per_rate,
        "latency_ms": {"p50": best["p50_ms"], "p99": best["p99_ms"]},
        "one_at_a_time_qps": one_qps,
        "served_vs_one_at_a_time": best["qps"] / one_qps,
        "equal_results_checked": len(sample),
        "e2e": {"value": ws * best["qps"], "unit": "queries/s", "h2d_bytes_per_step": 88 * nq,
                "d2h_bytes_per_step": sum(24 * q.k + 600 for q in qs)},
        "gpu_launches": None, "roofline": None,
        "cpu_baseline": {"value": cpu_qps, "unit": "queries/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {cpu_n} of the {nq} queries, serial C oracle, {cpu_s:.1f} s"},
        "clocks": clk,
    })
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rpq", choices=["rpq", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=4)
    ap.add_argument("--workload", default="medium", choices=sorted(WORKLOADS),
                    help="medium (default, the benchmark line), large, batched or served")
    ap.add_argument("--queries", type=int, default=0, help="use only the first Q queries of the workload")
    ap.add_argument("--autotune", type=int, default=1, help="run the library's autotuner first (1) or not (0)")
    ap.add_argument("--tune-queries", type=int, default=16, help="queries of the workload the autotuner times")
    ap.add_argument("--profile-only", type=int, default=0, metavar="Q",
                    help="load the workload, run its first Q queries once through rpq_search and exit "
                         "(a short command for ncu captures); prints no JSON line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_only:
        return profile_only(args.profile_only, args.workload)
    return run(args)


def profile_only(nq: int, workload: str = "medium") -> int:
    import torch
    import paper_2001_06770_b300 as rpq
    import rpqgen
    wl = WORKLOADS[workload]
    ds = rpqgen.make_dataset(wl["ds"])
    qs = rpqgen.workload_queries(wl["queries"], ds)[:nq]
    kg = rpq.KG.from_dataset(ds)
    for q in qs:
        kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
    torch.cuda.synchronize()
    kg.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
