"""Benchmark of the B300 radial-pattern keyword search (one JSON line on stdout).

Workload (N = 1, default): the large open-KG-shaped graph - Chung-Lu
(exponent 2.1), 5e7 nodes, 4e8 sampled edges (7.6e8 CSR entries, maximum
degree 638,167), int32 CSR both directions, Zipf(1.0) keywords over a 5M-word
vocabulary - with 256 queries issued one at a time (|C| = |M| = 3, keyword
ranks 100..20,000, k = 20, max depth 8).  One step = the 256 queries.

  value      queries/s with the query keyword ids already in device memory and
             results left there (rpq_search_device, CUDA graph per shape),
             CUDA events on the library's stream; the 3 GB adjacency is larger
             than L2 and L2 is also flushed between steps
  e2e        the same through rpq_search (host buffers in and out, one
             synchronous call per query), wall clock
  batched    the batched workload's mix (uneven shapes, head and tail
             keywords) on the same graph through rpq_search_batch, against the
             same queries one at a time, results compared
  roofline   the expansion kernel: algorithmic bytes / its device time,
             measured with CUDA events around each launch (profiling pass)
  cpu_baseline  the serial CPU oracle on a sample of the workload, one query
             per host core (threads sharing one prepared graph); every
             sampled result is compared with the GPU's (oracle_checked)

``--impl reference`` times the CPU oracle itself as the reference arm.
``--workload medium|batched|served`` runs the other configurations.
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
WORKLOAD_LARGE = ("large: Chung-Lu (exponent 2.1) 5e7 nodes, 4e8 sampled edges, symmetric int32 CSR; "
                  "256 RPQs one at a time, |C| = |M| = 3, ranks 100-20000, k=20, L=8")
REL_TOL = 1e-6   # S^r; node ids, S^c and S^m must be equal
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6400.0
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture)
# of every expansion launch of a workload's first queries, per workload, for
# the kernel source with this SHA-1 prefix; reported only while the
# expansion source is unchanged.
NCU_TRAFFIC = {
    # 8 queries of the large workload, one B300, every k_expand launch (80)
    "large": {"sha1": "56b9c58e3ee4", "queries": 8, "launches": 80, "dram_bytes": 24139829248},
}


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


def same_results(res, orc) -> bool:
    """A GPU result array equals the oracle's: node ids, S^c and S^m exactly,
    S^r within REL_TOL relative, same count and order."""
    return (len(res) == len(orc.nodes) and res["node"].tolist() == [int(x) for x in orc.nodes]
            and res["s_c"].tolist() == orc.s_c.tolist() and res["s_m"].tolist() == orc.s_m.tolist()
            and bool(np.allclose(res["s_r"], orc.s_r, rtol=REL_TOL, atol=0)))


class OracleLeg:
    """The serial CPU oracle on one dataset: its activation levels and the
    graph's transpose are built once (outside any timed region), then
    queries run one per thread on the host cores (each search is the serial
    oracle; the ctypes calls release the GIL, so the threads run in parallel
    and share one copy of the graph)."""

    def __init__(self, ds):
        import oracle
        t = time.perf_counter()
        self.act = oracle.dataset_activation(ds, detail=False)
        self.pg = oracle.PreparedGraph(ds, self.act.a)
        self.setup_s = time.perf_counter() - t

    def run(self, qs, threads=0):
        """(results, per-query seconds, wall seconds, threads) of the queries,
        query-parallel over `threads` threads (default: every host core)."""
        import oracle
        from concurrent.futures import ThreadPoolExecutor
        qs = list(qs)
        threads = max(1, min(threads or (os.cpu_count() or 1), max(len(qs), 1)))

        def one(q):
            t = time.perf_counter()
            r = oracle.search(None, None, q.central, q.marginal, q.k, q.max_depth, q.gamma,
                              w=getattr(q, "w", 0), product=getattr(q, "product", False), prepared=self.pg,
                              trace=False, subgraphs=False)
            return r, time.perf_counter() - t

        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=threads) as ex:
            out = list(ex.map(one, qs))
        wall = time.perf_counter() - t0
        return [r for r, _ in out], [d for _, d in out], wall, threads

    def check(self, qs, gpu_results, what="", threads=0):
        """Run the oracle on `qs` and assert that every GPU result equals it;
        returns the cpu_baseline record of that run."""
        res, per_q, wall, threads = self.run(qs, threads)
        for i, (g, o) in enumerate(zip(gpu_results, res)):
            if not same_results(g, o):
                raise AssertionError(f"{what} query {i}: GPU {g.tolist()} != oracle {list(zip(o.nodes.tolist(), o.s_c.tolist(), o.s_m.tolist(), o.s_r.tolist()))}")
        return {"value": len(qs) / wall, "unit": "queries/s", "cores": threads, "kind": "oracle",
                "per_query_s": {"mean": float(np.mean(per_q)), "max": float(np.max(per_q))},
                "wall_s": wall, "setup_s": self.setup_s}

    def close(self):
        self.pg.close()


def sample_indices(n, count):
    """`count` query indices spread evenly over n (all of them if count >= n)."""
    if count >= n:
        return list(range(n))
    return sorted(set(int(round(i * (n - 1) / max(count - 1, 1))) for i in range(count)))


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
    """The reference arm: the serial CPU oracle itself on this workload's
    queries, one query per host core at a time (threads sharing one prepared
    graph).  A step is one query of the workload (cycling through them); the W
    warm-up queries run first, then the K timed ones, each wave as wide as the
    host has cores."""
    ws, rank, _ = dist_init()
    if rank != 0:
        return 0
    import rpqgen
    wl = WORKLOADS[args.workload]
    ds = rpqgen.make_dataset(wl["ds"])
    qs = rpqgen.workload_queries(wl["queries"], ds)
    leg = OracleLeg(ds)
    order = [qs[i % len(qs)] for i in range(args.warmup + args.steps)]
    leg.run(order[:args.warmup])
    _, per_q, wall, threads = leg.run(order[args.warmup:])
    leg.close()
    qps = args.steps / wall
    line = {"impl": "reference", "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": wl["desc"], "step": "one query of the workload (cycling), "
                       f"{threads} queries at a time on {threads} host threads"},
            "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} timed queries of the {len(qs)} after {args.warmup} warm-up "
                                       f"queries, serial C oracle, one query per thread on {threads} threads "
                                       f"sharing one prepared graph (set-up {leg.setup_s:.0f} s untimed)",
                             "per_query_s": {"mean": float(np.mean(per_q)), "max": float(np.max(per_q))}},
            "host_cpu": host_cpu(),
            "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


WORKLOADS = {
    "medium": dict(ds="medium", queries="medium", mode="single", desc=WORKLOAD),
    "tiny": dict(ds="tiny", queries="tiny", mode="single",
                 desc="tiny: R-MAT 2^14 nodes, one RPQ (smoke and multi-process checks, not a bench line)"),
    "large": dict(ds="large", queries="large", mode="single", desc=WORKLOAD_LARGE),
    "cl_5m": dict(ds="cl_5m", queries="cl_5m", mode="single",
                  desc="cl_5m: Chung-Lu (exponent 2.1) 5e6 nodes, 4e7 sampled edges; the large workload's "
                       "queries (profiling case, not a bench line)"),
    "batched": dict(ds="large", queries="batched", mode="batch",
                    desc="batched: large graph; 4096 RPQs of uneven shape (|C| 2-6, |M| 0-8, head/tail keywords, "
                         "k in {5,10,20}, L=8) in one rpq_search_batch call"),
    "served": dict(ds="medium", queries="served", mode="serve",
                   desc="served: medium graph; 20000 RPQs (shapes as batched) arriving as a Poisson stream, "
                        "continuous batching under a 16 GB slot budget"),
}


DENSE_UNITS = 1 << 20   # a Glevel with at least this many work units (4 MB of adjacency) counts as dense


def level_bytes(r, n):
    """Algorithmic bytes of one Glevel (a record of rpq_profile_levels) for
    the expansion and for the frontier enqueue.  Expansion: 4 per work unit
    (the packed CSR entry), 1 per (column, edge) activation executed (the
    neighbour's visited byte), 2 per claim written (level byte and visited
    bit), 10 per item (record and column mask).  Enqueue: the frontier read
    (the n-bit bit map, or 4 bytes per queued node), per frontier node its
    row bounds (8), two level-index entries (4), its visited byte and one
    level byte per column, and the items and warp-tile starts it writes."""
    exp = 4 * r["units"] + r["e_act"] + 2 * r["claims"] + 10 * r["items"]
    fr = r["frontier"]
    scan = 4 * fr if r["flags"] & 8 else (n + 7) // 8
    enq = scan + fr * (13 + r["columns"]) + 10 * r["items"] + 4 * ((r["units"] + 127) // 128)
    return exp, enq


def expand_roofline(kg, qs, stats, workload="large"):
    """Profiling pass (kernels launched directly, CUDA events around each
    launch): device time per kernel class, and per Glevel the algorithmic
    bytes of the expansion and the enqueue against the measured HBM peak -
    over all launches, and over the dense levels alone.  The ncu DRAM bytes
    stored in NCU_TRAFFIC (per workload, for the expansion source they were
    captured with) are set beside the same launches' algorithmic bytes."""
    kg.set_profiling(True)
    kg.profile(reset=True)
    kg.profile_levels(reset=True)
    recs = []
    for i, q in enumerate(qs):
        kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)
        recs += [dict(r, query=i) for r in kg.profile_levels(reset=True)]
    prof = kg.profile(reset=True)
    kg.set_profiling(False)
    peak, peak_kind = hbm_peak()
    exp_ms, exp_launches = prof["expand"]
    total_ms = sum(v[0] for v in prof.values())

    def agg(rows, kind):
        ms = sum(r[f"{kind}_ms"] for r in rows)
        by = sum(level_bytes(r, kg.n)[0 if kind == "expand" else 1] for r in rows)
        ach = by / (ms / 1e3) / 1e9 if ms > 0 else 0.0
        return {"launches": len(rows), "ms": ms, "alg_bytes": by, "achieved": ach, "frac": ach / peak,
                "alg_bytes_per_launch": by / max(len(rows), 1), "avg_launch_us": 1e3 * ms / max(len(rows), 1)}

    expanded = [r for r in recs if r["flags"] & 1]
    dense = [r for r in expanded if r["units"] >= DENSE_UNITS]
    e_all, e_dense, q_all = agg(expanded, "expand"), agg(dense, "expand"), agg(recs, "enqueue")
    q_dense = agg([r for r in recs if r["frontier"] >= (1 << 18)], "enqueue")
    # DRAM bytes of the expansion launches of the workload's first queries,
    # from one ncu capture of the same kernel source (NCU_TRAFFIC), beside the
    # algorithmic bytes and device time of the same launches in this pass
    cap = NCU_TRAFFIC.get(workload)
    traffic = dram_gbs = traffic_ratio = None
    if cap and cap["sha1"] == expand_source_sha() and len(qs) >= cap["queries"]:
        same = [r for r in recs if r["query"] < cap["queries"]]     # every k_expand launch of those queries
        if len(same) == cap["launches"]:
            a = agg(same, "expand")
            traffic = cap["dram_bytes"] / cap["launches"]
            traffic_ratio = cap["dram_bytes"] / a["alg_bytes"] if a["alg_bytes"] else None
            dram_gbs = cap["dram_bytes"] / (a["ms"] / 1e3) / 1e9 if a["ms"] > 0 else None
    roof = {"bound": "hbm", "kernel": "k_expand", "achieved": e_all["achieved"], "peak": peak, "unit": "GB/s",
            "frac": e_all["frac"], "traffic": traffic, "peak_kind": peak_kind,
            "traffic_note": (f"ncu DRAM bytes per launch over the expansion launches of the first "
                             f"{cap['queries']} queries" if traffic else None),
            "traffic_over_alg_bytes": traffic_ratio,
            "dram_gbs": dram_gbs, "dram_frac": dram_gbs / peak if dram_gbs else None,
            "alg_bytes_per_launch": e_all["alg_bytes_per_launch"], "avg_launch_us": e_all["avg_launch_us"],
            "launches": e_all["launches"], "share_of_device_time": exp_ms / total_ms if total_ms else None,
            "dense": dict(e_dense, units_min=DENSE_UNITS,
                          share_of_expand_time=e_dense["ms"] / e_all["ms"] if e_all["ms"] else None),
            "enqueue": dict(q_all, kernel="k_enqueue", dense=dict(q_dense, frontier_min=1 << 18),
                            share_of_device_time=prof["enqueue"][0] / total_ms if total_ms else None)}
    return roof, {k: v[0] for k, v in prof.items()}


def step_transfer_bytes(qs):
    """Host-to-device and device-to-host bytes of the queries' host-API calls
    (the library reports the per-call sizes)."""
    import paper_2001_06770_b300 as rpq
    per = [rpq.transfer_bytes(q.k) for q in qs]
    return sum(h for h, _ in per), sum(d for _, d in per)


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
    tuned = kg.autotune(qs[:args.tune_queries], repeats=3) if args.autotune else kg.tuning()
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
    h2d, d2h = step_transfer_bytes(qs)            # query records in, control blocks with results out

    # batched: all queries in one rpq_search_batch call (concurrent slots)
    kg.search_batch(qs)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        kg.search_batch(qs)
    t_b = allmax(ws, time.perf_counter() - t0)
    batched = ws * nq * args.steps / t_b

    roof, kms = expand_roofline(kg, qs, stats, args.workload)
    # the batched workload's mix on the same graph (large only): one batch
    # call against the same queries one at a time, results compared
    mix = batched_mix(args, ws, ds, kg) if args.workload == "large" and args.mix_queries else None
    if rank != 0:
        return None
    # the oracle on a sample of the queries (one per host core, or all of
    # them on the medium graph); every sampled GPU result must equal it
    cores = os.cpu_count() or 1
    n_check = args.cpu_sample if args.cpu_sample >= 0 else (nq if kg.n <= (1 << 22) else max(8, cores))
    idx = sample_indices(nq, n_check)
    leg = OracleLeg(ds)
    cpu = leg.check([qs[i] for i in idx], [host_res[i] for i in idx], "one-at-a-time")
    checked = {"one_at_a_time": len(idx)}
    if mix is not None:
        midx = sample_indices(len(mix["queries"]), max(4, cores // 2))
        leg.check([mix["queries"][i] for i in midx], [mix["results"][i] for i in midx], "batched mix")
        checked["batched_mix"] = len(midx)
    leg.close()
    mc = raks_cpu_sample(ds, qs, 8) if args.raks_cpu else None
    line = base_line(args, ws, wl, value, t_dev / args.steps, args.steps)
    line.update({
        "config": {"workload": wl["desc"], "queries_per_step": nq, "n": kg.n, "m2": kg.m2, "abar": ds.abar,
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{ws}"},
        "gteps": e_act * ws * args.steps / t_dev / 1e9,
        "e_act_per_step": e_act,
        "e_act_skipped_per_step": sum(s["e_act_skipped"] for s in stats),
        "batched_qps": batched,
        "batched_mix": None if mix is None else {k: v for k, v in mix.items() if k not in ("queries", "results")},
        "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99))},
        "e2e": {"value": e2e, "unit": "queries/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roof,
        "kernel_ms_per_step": kms,
        "oracle_checked": checked,
        "cpu_baseline": dict(cpu, sample=f"{len(idx)} of the {nq} queries (evenly spaced), serial C oracle, "
                                         f"one query per thread on {cpu['cores']} threads sharing one prepared "
                                         f"graph; wall {cpu['wall_s']:.1f} s, set-up {cpu['setup_s']:.0f} s "
                                         f"untimed; every result equal to the GPU's"),
        "host_cpu": host_cpu(),
        "raks_cpu": None if mc is None else {
            "value": mc[0], "unit": "queries/s", "threads": mc[3], "kind": "paper's multi-core CPU search (OpenMP)",
            "sample": f"first {mc[2]} of the {nq} queries, {mc[1]:.1f} s"},
        "clocks": clk,
    })
    return line


def batched_mix(args, ws, ds, kg):
    """The first `--mix-queries` queries of the batched workload (uneven
    shapes, head and tail keywords) on the loaded graph: one rpq_search_batch
    call against the same queries one at a time; every result must agree."""
    import rpqgen
    mq = rpqgen.workload_queries("batched", ds)[:args.mix_queries]
    out = kg.search_batch(mq)                                   # warm-up and results
    assert all(st == 0 for _, _, st in out), "batch query failed"
    barrier(ws)
    t0 = time.perf_counter()
    out = kg.search_batch(mq)
    t_b = allmax(ws, time.perf_counter() - t0)
    pers = kg.search_batch(mq, persistent=True)                 # warm-up and results
    barrier(ws)
    t0 = time.perf_counter()
    pers = kg.search_batch(mq, persistent=True)
    t_p = allmax(ws, time.perf_counter() - t0)
    for i, ((b, _, _), (p, _, st)) in enumerate(zip(out, pers)):
        assert st == 0 and p.tobytes() == b.tobytes(), f"persistent-batch result differs on mix query {i}"
    barrier(ws)
    t0 = time.perf_counter()
    one = [kg.search(q.central, q.marginal, q.k, q.max_depth, q.gamma)[0] for q in mq]
    t_1 = allmax(ws, time.perf_counter() - t0)
    for i, (r, (b, _, _)) in enumerate(zip(one, out)):
        assert r.tobytes() == b.tobytes(), f"batched result differs from one-at-a-time on mix query {i}"
    return {"queries_per_call": len(mq), "batched_qps": ws * len(mq) / t_b, "one_at_a_time_qps": ws * len(mq) / t_1,
            "batched_vs_one_at_a_time": t_1 / t_b, "persistent_batch_qps": ws * len(mq) / t_p,
            "persistent_vs_slots": t_b / t_p, "equal_results_checked": len(mq),
            "e_act": sum(st["e_act_central"] + st["e_act_marginal"] for _, st, _ in out),
            "queries": mq, "results": one}


def run_batch(args, ws, rank, local, wl, ds, qs, kg):
    """All queries in one rpq_search_batch call per step; a sample is also run
    one at a time and must give identical results."""
    nq = len(qs)
    pers = args.batch_form == "persistent"
    res0 = kg.search_batch(qs, persistent=pers)
    assert all(st == 0 for _, _, st in res0), "batch query failed"
    sample = list(range(0, nq, max(1, nq // 128)))
    t0 = time.perf_counter()
    for i in sample:
        r, _ = kg.search(qs[i].central, qs[i].marginal, qs[i].k, qs[i].max_depth, qs[i].gamma)
        assert r.tobytes() == res0[i][0].tobytes(), f"batched result differs from one-at-a-time on query {i}"
    one_qps = len(sample) / (time.perf_counter() - t0)
    for _ in range(max(0, args.warmup - 1)):
        kg.search_batch(qs, persistent=pers)
    clocks = Clocks(local)
    barrier(ws)
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        out = kg.search_batch(qs, persistent=pers)
    t = allmax(ws, time.perf_counter() - t0)
    clk = clocks.stop()
    value = ws * nq * args.steps / t
    # the other batch form, one pass on the same queries (same results)
    t0 = time.perf_counter()
    other = kg.search_batch(qs, persistent=not pers)
    t_other = allmax(ws, time.perf_counter() - t0)
    for i, ((a, _, _), (b, _, st)) in enumerate(zip(out, other)):
        assert st == 0 and a.tobytes() == b.tobytes(), f"batch forms differ on query {i}"
    stats = [st for _, st, _ in out]
    e_act = sum(s["e_act_central"] + s["e_act_marginal"] for s in stats)
    sstats = [stats[i] for i in sample]
    roof, kms = expand_roofline(kg, [qs[i] for i in sample], sstats, args.workload)
    if rank != 0:
        return None
    cores = os.cpu_count() or 1
    idx = sample_indices(nq, args.cpu_sample if args.cpu_sample >= 0 else max(8, cores))
    leg = OracleLeg(ds)
    cpu = leg.check([qs[i] for i in idx], [out[i][0] for i in idx], "batched")
    leg.close()
    line = base_line(args, ws, wl, value, t / args.steps, args.steps)
    line.update({
        "config": {"workload": wl["desc"], "queries_per_step": nq, "n": kg.n, "m2": kg.m2, "abar": ds.abar,
                   "slots": kg.tuning()["batch_slots"], "l2": "inputs larger than L2 (3 GB adjacency)", "parallelism": f"replicas x{ws}"},
        "gteps": e_act * ws * args.steps / t / 1e9,
        "one_at_a_time_qps": one_qps,
        "batched_vs_one_at_a_time": value / (ws * one_qps),
        "batch_form": args.batch_form,
        ("slots_qps" if pers else "persistent_qps"): ws * nq / t_other,
        "equal_results_checked": len(sample),
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": step_transfer_bytes(qs)[0],
                "d2h_bytes_per_step": step_transfer_bytes(qs)[1]},
        "gpu_launches": (1 if pers else sum(s["kernels"] for s in stats)) * args.steps,   # persistent: one launch per step
        "roofline": roof, "kernel_ms_per_step_sample": kms,
        "oracle_checked": {"batched": len(idx)},
        "cpu_baseline": dict(cpu, sample=f"{len(idx)} of the {nq} queries (evenly spaced), serial C oracle, "
                                         f"one query per thread on {cpu['cores']} threads sharing one prepared "
                                         f"graph; wall {cpu['wall_s']:.1f} s; every result equal to the GPU's"),
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
    served = {}

    def serve_at(rate, below=False):
        arr = rpqgen.poisson_arrivals(nq, rate, seed=7)
        res, lat, status, wall = srv.replay(qs, arr)
        assert (status == 0).all()
        for i in sample:
            assert res[i].tobytes() == alone[i].tobytes(), f"served result differs from alone on query {i}"
        if not served:
            served.update({i: res[i] for i in sample})
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
    srv_info = srv.info()           # pools, and the most queries that ran at once
    srv.close()
    if rank != 0:
        return None
    best = max((r for r in per_rate if not r["below_capacity"]), key=lambda r: r["qps"])
    # the served results of the sampled queries against the oracle
    leg = OracleLeg(ds)
    cpu = leg.check([qs[i] for i in sample], [served[i] for i in sample], "served")
    leg.close()
    line = base_line(args, ws, wl, ws * best["qps"], best["wall_s"], 1)
    line.update({
        "config": {"workload": wl["desc"], "queries": nq, "n": kg.n, "m2": kg.m2, "budget_bytes": 16 << 30,
                   "l2": "inputs larger than L2", "parallelism": f"replicas x{ws}"},
        "server": {k: v for k, v in srv_info.items() if k not in ("running", "waiting")},
        "per_rate": per_rate,
        "latency_ms": {"p50": best["p50_ms"], "p99": best["p99_ms"]},
        # service latency: the stream at 80% of the measured capacity
        "latency_ms_below_capacity": {k: v for k, v in per_rate[-1].items() if k != "below_capacity"},
        "one_at_a_time_qps": one_qps,
        "served_vs_one_at_a_time": best["qps"] / one_qps,
        "equal_results_checked": len(sample),
        "e2e": {"value": ws * best["qps"], "unit": "queries/s", "h2d_bytes_per_step": step_transfer_bytes(qs)[0],
                "d2h_bytes_per_step": step_transfer_bytes(qs)[1]},
        "gpu_launches": None, "roofline": None,
        "oracle_checked": {"served": len(sample)},
        "cpu_baseline": dict(cpu, sample=f"{len(sample)} of the {nq} queries (evenly spaced), serial C oracle, "
                                         f"one query per thread on {cpu['cores']} threads sharing one prepared "
                                         f"graph; wall {cpu['wall_s']:.1f} s; every served result equal to it"),
        "clocks": clk,
    })
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rpq", choices=["rpq", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=-1,
                    help="queries the oracle checks (-1: every query on medium, one per host core on large)")
    ap.add_argument("--raks-cpu", type=int, default=1, help="time the paper's OpenMP CPU search on 8 queries")
    ap.add_argument("--batch-form", default="slots", choices=["slots", "persistent"],
                    help="batched workload: per-query graphs on concurrent slots, or the whole batch in one "
                         "persistent kernel fed by a device work queue (the other form is timed once beside it)")
    ap.add_argument("--mix-queries", type=int, default=512,
                    help="large workload: queries of the batched mix run batched and one at a time")
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS),
                    help="large (default, the benchmark line), medium, batched or served")
    ap.add_argument("--queries", type=int, default=0, help="use only the first Q queries of the workload")
    ap.add_argument("--autotune", type=int, default=1, help="run the library's autotuner first (1) or not (0)")
    ap.add_argument("--tune-queries", type=int, default=32, help="queries of the workload the autotuner times")
    ap.add_argument("--profile-only", type=int, default=0, metavar="Q",
                    help="load the workload, run its first Q queries once through rpq_search and exit "
                         "(a short command for ncu captures); prints no JSON line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_only:
        return profile_only(args.profile_only, args.workload)
    return run(args)


def profile_only(nq: int, workload: str = "large") -> int:
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
