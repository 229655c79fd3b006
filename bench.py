"""Benchmark: BGP queries/s with p50/p99 latency on seeded R-MAT RDF graphs
resident on one B300, the triple-scan roofline and the CPU oracle beside
them. Prints one JSON line on rank 0.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rmat26]
                    [--impl gsmart|reference] [--mode plain|scan|batched|served|query]

Default (the scale-26, 1.07e9-triple graph): the bandwidth workload's
constant-free cycles, each of which starts with a triple scan over all
2.1e9 labels. The headline is served queries/s under Poisson arrivals at
20,000 offered queries/s (a step is 256 arrivals); the same queries one at
a time (plain) and as one batch are reported beside it, and `e2e` is the
served replay with every answer copied into pinned host memory.
`--workload rmat22` is the mid configuration: its 32 mixed queries one at
a time per step, with the answer rows fetched for `e2e`. With N > 1
(torchrun) every rank holds its own copy of the graph and runs the whole
workload (replicas: queries are independent, there is no exchange).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rdfgen  # noqa: E402


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rmat26")
    ap.add_argument("--impl", default="gsmart", choices=["gsmart", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=20.0,
                    help="budget of the CPU oracle sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--mode", default="plain",
                    choices=["plain", "scan", "batched", "served", "query", "paths", "lspm"],
                    help="plain: the workload's queries one at a time (the headline line); "
                         "scan: the triple scan alone; batched: the batched workload "
                         "(rmat24: 4,096 queries in one launch) against one at a time; "
                         "served: Poisson arrivals into the server on the scale-26 graph; "
                         "query: the workload queries --query picks, one at a time (for "
                         "profiling single kernels); paths: per-path trees against the "
                         "path-linearized tree; lspm: each query on its per-query LSpM "
                         "against the full store")
    ap.add_argument("--queries", type=int, default=0,
                    help="batched mode: number of queries (0: the workload's)")
    ap.add_argument("--query", default="0",
                    help="query mode: comma-separated indices into the workload's queries")
    ap.add_argument("--family", default="default", choices=["default", "bandwidth"],
                    help="query mode: the workload's own queries, or the bandwidth family's "
                         "copy for its graph (rdfgen/<workload>_bandwidth.txt)")
    ap.add_argument("--trace", action="store_true",
                    help="query mode: also report each query's device ms per phase "
                         "(setup + triple scan, each level, enumeration; grid-path queries)")
    ap.add_argument("--batch", action="store_true",
                    help="query mode: evaluate the selected queries as one batch per round")
    return ap.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0}, "fallback"


class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            # a short timed region may end before nvidia-smi's first line
            t0 = time.time()
            while len(self.lines) < 1 and time.time() - t0 < 2.0:
                time.sleep(0.02)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_rate(local_ms: float, units_per_rank: int, world: int, dist=None, device="cuda"):
    """Whole-job rate of a replicated step: the units every rank processed
    divided by the slowest rank's time (max over ranks). Returns (rate per
    second, max milliseconds)."""
    t_ms = float(local_ms)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([t_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    return world * units_per_rank / (t_ms / 1000.0), t_ms


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _workload(name, family="default"):
    w = rdfgen.WORKLOADS[name]
    s, p, o = rdfgen.graph(w)
    if name == "rmat26" or family == "bandwidth":   # the bandwidth family's stored queries
        return w, (s, p, o), rdfgen.bandwidth_workload(w)
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    qs = rdfgen.queries(w, sm)
    sm.close()
    return w, (s, p, o), qs


BANDWIDTH_METRIC = ("BGP queries/s (served: Poisson arrivals, continuous batching; plain and "
                    "batched beside), triple-scan HBM GB/s")
PER_STEP = 256           # arrivals per step of the served headline
TOP_RATE = 20000         # its offered queries/s


def _bandwidth_config(w, M, n_queries, ws):
    """config of the scale-26 line, the same for both arms."""
    N = w.n_vertices
    return {"workload": w.name, "scale": w.scale, "triples_drawn": w.n_edges, "triples": int(M),
            "predicates": w.n_preds, "queries": n_queries,
            "query_mix": "constant-free 3-/4-cycles, with and without a pendant edge "
                         "(rdfgen/rmat26_bandwidth.txt)",
            "offered_qps": TOP_RATE, "arrivals_per_step": PER_STEP,
            "memory_budget_bytes": 40 << 30,
            "l2": "inputs larger than L2 (graph %.1f GB; every query scans 2.1e9 labels)"
                  % ((8 * (N + 1) + 16 * M) / 1e9),
            "parallelism": "replicas" if ws > 1 else "single"}


def _cpu_baseline(w, triples, qs, budget_s):
    """The oracle as it stands, on all host cores, on a bounded sample."""
    import oracle
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ix = oracle.Index(*triples, w.n_vertices, w.n_preds)
    build_s = time.perf_counter() - t0
    done, rows, t0 = 0, 0, time.perf_counter()
    for q in qs:
        rows += len(ix.eval(q.patterns, threads=cores))
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": "first %d of %d queries of %s, one at a time, %d answer rows; "
                      "index build %.1f s excluded" % (done, len(qs), w.name, rows, build_s)}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    w, triples, qs = _workload(args.workload)
    import oracle
    cores = os.cpu_count() or 1
    ix = oracle.Index(*triples, w.n_vertices, w.n_preds)
    # each step: a bounded prefix of the query list, sized so the run ends in minutes
    budget = max(2.0, 120.0 / max(1, args.steps + args.warmup))
    n_q = len(qs)
    t0 = time.perf_counter()
    for i, q in enumerate(qs):
        ix.eval(q.patterns, threads=cores)
        if time.perf_counter() - t0 > budget:
            n_q = i + 1
            break
    sample = qs[:n_q]
    for _ in range(args.warmup):
        for q in sample:
            ix.eval(q.patterns, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for q in sample:
            ix.eval(q.patterns, threads=cores)
    dt = time.perf_counter() - t0
    v = args.steps * len(sample) / dt
    desc = "first %d of %d queries of %s per step" % (len(sample), len(qs), w.name)
    if w.name == "rmat26":
        metric, config = BANDWIDTH_METRIC, _bandwidth_config(w, len(ix), len(qs), ws)
    else:
        metric = "BGP queries/s (plain, one at a time)"
        config = {"workload": w.name, "scale": w.scale, "triples_drawn": w.n_edges,
                  "predicates": w.n_preds, "queries": len(qs)}
    print(json.dumps({
        "impl": "reference", "metric": metric, "value": v,
        "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": v, "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_gsmart(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    import paper_2106_14038_b300 as gs

    def barrier():
        if dist is not None:
            dist.barrier()

    w, triples, qs = _workload(args.workload)
    g = gs.Graph(*triples, w.n_vertices, w.n_preds)
    stream = torch.cuda.current_stream()
    plans = None
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 126 MB L2

    def step(fetch: bool, lat=None, out_bufs=None, diag=None):
        launches, d2h, h2d = 0, 0, 0
        for i, q in enumerate(qs):
            t0 = time.perf_counter()
            plan = g.plan(q.patterns)
            r = g.eval(plan, stream)
            n, k = r.info()
            if fetch:
                buf = out_bufs[i]
                r.fetch(sort=False, out=buf[: n * k].view(n, k).numpy())
                d2h += 4 * n * k
                h2d += q.patterns.nbytes
            t1 = time.perf_counter()
            if lat is not None:
                lat.append(t1 - t0)
            dev_ms, nl = r.stats()
            launches += nl
            if diag is not None:
                diag.append((q.shape, n, nl, dev_ms, 1000 * (t1 - t0)))
            r.close()
            plan.close()
        return launches, h2d, d2h

    # pinned host buffers for the end-to-end answers (sized by one untimed run)
    sizes = []
    for q in qs:
        r = g.eval(q.patterns, stream)
        n, k = r.info()
        sizes.append(max(1, n * k))
        r.close()
    out_bufs = [torch.empty(sz, dtype=torch.int32, pin_memory=True) for sz in sizes]

    for _ in range(args.warmup):
        step(False)
    diag = []
    step(False, diag=diag)
    if rank == 0:
        for d in diag:
            print("query %-12s rows %10d launches %3d device %.3f ms host %.3f ms" % d,
                  file=sys.stderr)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat = []
    step_ms = []
    launches = 0
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            barrier()
            torch.cuda.synchronize()
            ev0.record(stream)
            launches, _, _ = step(False, lat)
            ev1.record(stream)
            torch.cuda.synchronize()
            barrier()
            step_ms.append(ev0.elapsed_time(ev1))
    clocks = clk.summary()
    value, t_ms = aggregate_rate(float(np.sum(step_ms)), len(qs) * args.steps, ws, dist)

    # batched: the same queries in one persistent launch per step, under the
    # configuration the native autotuner picks on them (untimed)
    tune_plans = [g.plan(q.patterns) for q in qs]
    bcfg, tune_ms = g.autotune_batch(tune_plans, stream)
    for pl in tune_plans:
        pl.close()

    def batch_step():
        plans = [g.plan(q.patterns) for q in qs]
        b = g.eval_batch(plans, stream, config=bcfg)
        rows = b.rows()
        st = b.stats()
        b.close()
        for pl in plans:
            pl.close()
        return rows, st

    for _ in range(args.warmup):
        batch_step()
    b_ms, b_stats = [], None
    for _ in range(args.steps):
        flush.fill_(1)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        brows, b_stats = batch_step()
        torch.cuda.synchronize()
        b_ms.append(1000 * (time.perf_counter() - t0))
    b_value, b_total = aggregate_rate(float(np.sum(b_ms)), len(qs) * args.steps, ws, dist)
    batched = {"value": b_value, "unit": "queries/s",
               "ms_per_step": b_total / args.steps, "device_ms_last": b_stats[0],
               "kernel_launches_per_step": b_stats[1], "grid_path_queries": b_stats[2],
               "rows_per_step": int(np.sum(brows)),
               "config": bcfg.as_dict(), "autotune_best_ms": tune_ms,
               "timing": "host wall clock per step (plan + one batch launch + counts)"}

    # served: Poisson arrivals into the continuous-batching server
    served = served_rates(g, qs, [200, 2000, 20000], 6000, 3000 + args.steps, bcfg)

    # end to end: same step with answers copied into pinned host memory
    e2e_ms = []
    for _ in range(args.steps):
        flush.fill_(1)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, h2d, d2h = step(True, None, out_bufs)
        torch.cuda.synchronize()
        e2e_ms.append(1000 * (time.perf_counter() - t0))
    e2e_value, _ = aggregate_rate(float(np.sum(e2e_ms)), len(qs) * args.steps, ws, dist)

    # triple scan (Eq. 17 / Eq. 21 over the whole matrix): the bandwidth kernel
    peaks, which = _peaks()
    preds = [1, 2, 3, 1, 2]
    dirs = [0, 0, 0, 1, 1]
    words = (w.n_vertices + 31) // 32
    out = torch.empty(words, dtype=torch.int32, device="cuda")
    for _ in range(3):
        g.scan(preds, dirs, out=out)
    n_scan = 20
    se0, se1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    scan_ms = 0.0
    for _ in range(n_scan):
        flush.fill_(1)
        # ~2 ms on the device: the host enqueues the scan meanwhile, so no
        # host delay falls between the two events
        torch.cuda._sleep(4000000)
        se0.record(stream)
        g.scan(preds, dirs, out=out)
        se1.record(stream)
        torch.cuda.synchronize()
        scan_ms += se0.elapsed_time(se1)
    scan_ms /= n_scan
    N, M = w.n_vertices, g.n_triples
    alg_bytes = 2 * (4 * (N + 1) + 4 * M) + N // 8
    achieved = alg_bytes / (scan_ms / 1000.0) / 1e9
    roof = {"kernel": "triple-scan call (gs_scan_candidates: k_scan_zero + k_scan over both "
                      "orientations + k_scan_eval)",
            "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "peak_source": which,
            "traffic": _scan_traffic(w.name), "algorithmic_bytes": alg_bytes,
            "ms_per_launch": scan_ms}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = _cpu_baseline(w, triples, qs, args.cpu_seconds)

    if rank == 0:
        lat_ms = 1000 * np.array(lat)
        print(json.dumps({
            "metric": "BGP queries/s (plain, one at a time)", "value": value,
            "unit": "queries/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": w.name, "scale": w.scale, "triples_drawn": w.n_edges,
                       "triples": M, "predicates": w.n_preds, "queries": len(qs),
                       "l2": "flushed before every step (256 MiB write); graph %.2f GB > L2"
                             % ((8 * (N + 1) + 16 * M) / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "e2e": {"value": e2e_value, "unit": "queries/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "batched": batched,
            "served": served,
            "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": launches * args.steps,
        }), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one triple-scan
# call (k_scan_zero + k_scan + k_scan_eval) from one ncu capture, with the
# sha1 prefix of the scan source the counters were taken on; the summary is
# in profiles/. A changed kernel reports null until it is captured again.
SCAN_TRAFFIC = {
    "rmat22": ("f675e7461d73", 617415936),
    "rmat26": ("f675e7461d73", 10649202944),
}


def _scan_traffic(workload):
    entry = SCAN_TRAFFIC.get(workload)
    if not entry or entry[1] is None:
        return None
    src = os.path.join(ROOT, "paper_2106_14038_b300", "csrc", "gs_scan.cu")
    with open(src, "rb") as f:
        sha = hashlib.sha1(f.read()).hexdigest()
    return entry[1] if sha.startswith(entry[0]) else None


def served_rates(g, qs, rates, max_queries, seed, batch_cfg=None):
    """Poisson arrivals of the workload's queries (cycled) into the
    continuous-batching server, one run per offered rate, driven by the
    library's native replay loop. Latency runs from each query's scheduled
    arrival to its completion as the server's worker sees it; achieved q/s =
    queries / (last completion - first arrival)."""
    import paper_2106_14038_b300 as gs
    plans = [g.plan(q.patterns) for q in qs]
    out = []
    for rate in rates:
        n = int(min(max_queries, max(100, rate)))          # about one second of arrivals
        rng = np.random.default_rng(seed + int(rate))
        sched = np.cumsum(rng.exponential(1.0 / rate, n))
        srv = gs.Server(g, batch=batch_cfg)
        lat_us, done_s = srv.replay(plans, sched)
        completed, batches, peak = srv.stats()
        srv.stop()
        span = float(done_s.max() - sched[0])
        out.append({"offered_qps": rate, "queries": n, "achieved_qps": n / span,
                    "p50_ms": float(np.percentile(lat_us, 50) / 1e3),
                    "p99_ms": float(np.percentile(lat_us, 99) / 1e3),
                    "batches": batches, "peak_admitted_bytes": peak})
    for pl in plans:
        pl.close()
    return out


def run_scan_only(args):
    """The triple scan (Eq. 17 / Eq. 21 over the whole matrix) timed alone
    on the workload graph: the query's grouped predicate set is the root
    group of a constant-free star (three out-predicates, two in-predicates,
    the most frequent ones)."""
    import torch
    torch.cuda.set_device(0)
    import paper_2106_14038_b300 as gs
    w = rdfgen.WORKLOADS[args.workload]
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    del s, p, o
    preds, dirs = [1, 2, 3, 1, 2], [0, 0, 0, 1, 1]
    words = (w.n_vertices + 31) // 32
    out = torch.empty(words, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        g.scan(preds, dirs, out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    with Clocks(0) as clk:
        for _ in range(args.steps):
            torch.cuda.synchronize()
            flush.fill_(1)
            # ~2 ms on the device: the host enqueues the scan meanwhile, so no
            # host delay falls between the two events
            torch.cuda._sleep(4000000)
            e0.record(stream)
            g.scan(preds, dirs, out=out)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
    peaks, which = _peaks()
    N, M = w.n_vertices, g.n_triples
    alg = 2 * (4 * (N + 1) + 4 * M) + N // 8
    t = float(np.mean(ms))
    gbs = alg / (t / 1000.0) / 1e9
    print(json.dumps({
        "metric": "triple-scan HBM GB/s", "value": gbs, "unit": "GB/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "ms_min": float(np.min(ms)), "ms_median": float(np.median(ms)),
        "config": {"workload": w.name, "scale": w.scale, "triples": M, "predicates": w.n_preds,
                   "group": {"preds": preds, "dirs": dirs},
                   "l2": "flushed before every step (256 MiB write)"},
        "roofline": {"kernel": "triple-scan call (k_scan_zero + k_scan over both orientations "
                               "+ k_scan_eval)", "bound": "hbm", "achieved": gbs,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                     "peak_source": which, "peak_nominal": NOMINAL_HBM_GBS,
                     "frac_nominal": gbs / NOMINAL_HBM_GBS, "traffic": _scan_traffic(w.name),
                     "algorithmic_bytes": alg},
        "clocks": clk.summary(), "gpu_launches": 3 * args.steps,
    }), flush=True)


def run_batched(args):
    """The batched workload: its queries evaluated in one gs_eval_batch per
    step (autotuned on a sample, untimed) against the same queries one at a
    time; both through the C ABI with answers counted on the device."""
    import torch
    torch.cuda.set_device(0)
    import paper_2106_14038_b300 as gs
    name = args.workload if args.workload not in ("rmat22", "rmat26") else "rmat24"
    w = rdfgen.WORKLOADS[name]
    t0 = time.perf_counter()
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    nq = args.queries or w.n_queries
    stored = os.path.join(ROOT, "tests", "golden", "rmat24_batched.txt")
    if name == "rmat24" and os.path.exists(stored):
        # selected by exact answer count in [t/2, 2t] (the file's header)
        qs = rdfgen.load_queries(stored)[:nq]
        selection = "exact count in [t/2, 2t], t log-uniform in [1, 1e6] (%s)" % os.path.basename(stored)
    else:
        sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
        qs = rdfgen.batched_queries(w, sm, nq)
        sm.close()
        selection = "spanning-tree bound at most t (an upper bound on the count)"
    del s, p, o
    prep_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    sample = [g.plan(q.patterns) for q in qs[: min(512, len(qs))]]
    bcfg, tune_ms = g.autotune_batch(sample, stream)
    for pl in sample:
        pl.close()

    def batch_step():
        plans = [g.plan(q.patterns) for q in qs]
        b = g.eval_batch(plans, stream, config=bcfg)
        rows = b.rows()
        st = b.stats()
        b.close()
        for pl in plans:
            pl.close()
        return rows, st

    for _ in range(args.warmup):
        batch_step()
    b_ms, rows, st = [], None, None
    with Clocks(0) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            rows, st = batch_step()
            torch.cuda.synchronize()
            b_ms.append(1000 * (time.perf_counter() - t1))
    # one at a time: the same queries, one warm-up pass over a slice, one timed pass
    for q in qs[:64]:
        r = g.eval(q.patterns, stream)
        r.info()
        r.close()
    flush.fill_(1)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    prow = 0
    for q in qs:
        plan = g.plan(q.patterns)
        r = g.eval(plan, stream)
        prow += r.info()[0]
        r.close()
        plan.close()
    torch.cuda.synchronize()
    plain_ms = 1000 * (time.perf_counter() - t1)
    total_rows = int(np.sum(rows))
    assert prow == total_rows, (prow, total_rows)
    # with the stored selection, every query's row count is its oracle count
    counts_match = None
    if selection.startswith("exact"):
        counts_match = bool(np.array_equal(np.asarray(rows, np.int64),
                                           np.array([int(q.bound) for q in qs], np.int64)))
    t_ms = float(np.mean(b_ms))
    bounds = np.array([q.bound for q in qs])
    print(json.dumps({
        "metric": "BGP queries/s (batched: all queries in one launch per step)",
        "value": len(qs) / (t_ms / 1000.0), "unit": "queries/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": w.name, "scale": w.scale, "triples": g.n_triples,
                   "predicates": w.n_preds, "queries": len(qs),
                   "selection": selection,
                   "count_quantiles": [float(x) for x in np.quantile(bounds, [0, .1, .5, .9, 1])],
                   "counts_match_oracle": counts_match,
                   "l2": "flushed before every step (256 MiB write)",
                   "setup_s": prep_s},
        "batched": {"config": bcfg.as_dict(), "autotune_best_ms_on_512": tune_ms,
                    "grid_path_queries": st[2], "kernel_launches_per_step": st[1],
                    "rows_per_step": total_rows, "device_ms_last": st[0]},
        "plain": {"value": len(qs) / (plain_ms / 1000.0), "unit": "queries/s",
                  "ms_per_step": plain_ms, "rows": prow},
        "clocks": clk.summary(), "gpu_launches": st[1] * args.steps,
    }), flush=True)


def run_served(args):
    """The served configuration: the scale-26 graph resident, Poisson
    arrivals at 200 / 2,000 / 20,000 q/s of a query mix sampled on it
    (the batched workload's sampler: 2..10 shape vertices, 1..2 constants,
    log-uniform targets), admission by the server's memory budget; the same
    queries one at a time for comparison."""
    import torch
    torch.cuda.set_device(0)
    import paper_2106_14038_b300 as gs
    name = args.workload if args.workload != "rmat22" else "rmat26"
    w = rdfgen.WORKLOADS[name]
    t0 = time.perf_counter()
    s, p, o = rdfgen.graph(w)
    g = gs.Graph(s, p, o, w.n_vertices, w.n_preds)
    sm = rdfgen.Sampler(s, p, o, w.n_vertices, w.n_preds)
    del s, p, o
    wq = rdfgen.Workload(w.name, w.scale, w.n_edges, w.n_preds, w.zipf_s, w.graph_seed,
                         w.query_seed + 100, args.queries or 256, w.cap)
    qs = rdfgen.batched_queries(wq, sm)
    sm.close()
    prep_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    plans = [g.plan(q.patterns) for q in qs]
    bcfg, _ = g.autotune_batch(plans[:128], stream)
    # one at a time
    for q in qs[:32]:
        r = g.eval(q.patterns, stream)
        r.info()
        r.close()
    lat = []
    t1 = time.perf_counter()
    for pl in plans:
        a = time.perf_counter()
        r = g.eval(pl, stream)
        r.info()
        r.close()
        lat.append(time.perf_counter() - a)
    plain_s = time.perf_counter() - t1
    for pl in plans:
        pl.close()
    with Clocks(0) as clk:
        served = served_rates(g, qs, [200, 2000, 20000], 6000, 5000, bcfg)
    lat_ms = 1000 * np.array(lat)
    top = max(served, key=lambda x: x["achieved_qps"])
    print(json.dumps({
        "metric": "BGP queries/s (served: Poisson arrivals, continuous batching)",
        "value": top["achieved_qps"], "unit": "queries/s", "n_gpus": 1, "steps": 1,
        "warmup": 1, "ms_per_step": 1000.0 * top["queries"] / top["achieved_qps"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": w.name, "scale": w.scale, "triples": g.n_triples,
                   "predicates": w.n_preds, "queries": len(qs), "setup_s": prep_s,
                   "memory_budget_bytes": 40 << 30},
        "served": served, "batch_config": bcfg.as_dict(),
        "plain": {"value": len(qs) / plain_s, "unit": "queries/s",
                  "p50_ms": float(np.percentile(lat_ms, 50)),
                  "p99_ms": float(np.percentile(lat_ms, 99))},
        "clocks": clk.summary(),
    }), flush=True)


def run_query(args):
    """Selected queries of the plain workload, one at a time: W untimed
    rounds, then K rounds; one line with each query's mean device time."""
    import torch
    torch.cuda.set_device(0)
    import paper_2106_14038_b300 as gs
    w, triples, qs = _workload(args.workload, args.family)
    g = gs.Graph(*triples, w.n_vertices, w.n_preds)
    sel = [int(x) for x in args.query.split(",")]
    stream = torch.cuda.current_stream()
    if args.batch:
        plans = [g.plan(qs[i].patterns) for i in sel]
        ms, launches = [], 0
        for rep in range(args.warmup + args.steps):
            b = g.eval_batch(plans, stream)
            rows = b.rows()
            st = b.stats()
            if rep >= args.warmup:
                ms.append(st[0])
                launches += st[1]
            scans = b.scans()
            b.close()
        print(json.dumps({
            "metric": "device ms per batch", "unit": "ms", "higher_is_better": False,
            "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
            "config": {"workload": w.name, "family": args.family, "queries": sel},
            "device_ms": float(np.mean(ms)),
            "rows": [int(x) for x in rows], "triple_scans": scans[0], "gpu_launches": launches,
        }), flush=True)
        return
    dev = {i: [] for i in sel}
    info = {}
    phases = {i: [] for i in sel}
    launches = 0
    if args.trace:
        g.set_trace(True)
    for rep in range(args.warmup + args.steps):
        for i in sel:
            plan = g.plan(qs[i].patterns)
            r = g.eval(plan, stream)
            n, k = r.info()
            ms, nl = r.stats()
            if rep >= args.warmup:
                dev[i].append(ms)
                launches += nl
                if args.trace:
                    try:
                        phases[i].append(r.phases())
                    except gs.GsError:
                        pass
            if rep == 0:
                try:
                    tree = r.tree()
                except gs.GsError:
                    tree = None
                info[i] = (qs[i].shape, n, nl, tree, g.estimate(plan))
            r.close()
            plan.close()
    print(json.dumps({
        "metric": "device ms per query", "unit": "ms", "higher_is_better": False,
        "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
        "config": {"workload": w.name, "family": args.family, "queries": sel},
        "queries": [{"index": i, "shape": info[i][0], "rows": info[i][1], "launches": info[i][2],
                     "tree_nodes": info[i][3], "estimate_bytes": info[i][4][0],
                     "estimate_rows": info[i][4][1], "device_ms": float(np.mean(dev[i])),
                     "phases_ms": ([float(x) for x in np.mean(np.array(phases[i]), axis=0)]
                                   if phases[i] else None)}
                    for i in sel],
        "gpu_launches": launches,
    }), flush=True)


def run_bandwidth(args):
    """The bandwidth-bound configuration (the default line): the scale-26
    graph resident; the constant-free cycles of rdfgen/rmat26_bandwidth.txt,
    each starting with a triple scan over all 2.1e9 labels. Headline: served
    q/s under Poisson arrivals at the top offered rate (a step = 256
    arrivals), with p50/p99; beside it the lower offered rates, the same
    queries one at a time (plain) and as one batch, the end-to-end replay
    with every answer fetched into pinned host memory, the triple-scan
    roofline and the oracle on the host cores."""
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    import paper_2106_14038_b300 as gs

    def barrier():
        if dist is not None:
            dist.barrier()

    w = rdfgen.WORKLOADS[args.workload]
    t_setup = time.perf_counter()
    triples = rdfgen.graph(w)
    g = gs.Graph(*triples, w.n_vertices, w.n_preds)
    qs = rdfgen.bandwidth_workload(w)
    plans = [g.plan(q.patterns) for q in qs]
    setup_s = time.perf_counter() - t_setup
    stream = torch.cuda.current_stream()
    N, M = w.n_vertices, g.n_triples

    # plain: one query at a time (plan + evaluation + answer count)
    def plain_pass(lat=None):
        nl = 0
        for q in qs:
            t0 = time.perf_counter()
            plan = g.plan(q.patterns)
            r = g.eval(plan, stream)
            r.info()
            if lat is not None:
                lat.append(time.perf_counter() - t0)
            nl += r.stats()[1]
            r.close()
            plan.close()
        return nl
    for _ in range(args.warmup):
        plain_pass()
    lat, pl_ms = [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        torch.cuda.synchronize()
        ev0.record(stream)
        plain_pass(lat)
        ev1.record(stream)
        torch.cuda.synchronize()
        pl_ms.append(ev0.elapsed_time(ev1))
    plain_q, _ = aggregate_rate(float(np.sum(pl_ms)), len(qs) * args.steps, ws, dist)
    lat_ms = 1000 * np.array(lat)
    rows = [int(g.eval(pl, stream).info()[0]) for pl in plans]
    # one traced pass (untimed): device ms per phase of each query, setup +
    # triple scan, the binding-tree levels and the enumeration
    g.set_trace(True)
    phases = []
    for pl in plans:
        r = g.eval(pl, stream)
        r.info()
        try:
            ph = r.phases()
            phases.append((ph[0], float(sum(ph[1:-1])), ph[-1]))
        except gs.GsError:   # a query the single-CTA kernel finished has none
            pass
        r.close()
    g.set_trace(False)
    phase_summary = None
    if phases:
        a = np.array(phases)
        phase_summary = {"queries": len(phases), "setup_and_scan_ms": float(a[:, 0].mean()),
                         "levels_ms": float(a[:, 1].mean()), "enumerate_ms": float(a[:, 2].mean()),
                         "how": "one traced pass, untimed: CUDA events between the phases "
                                "of each query (mean over queries)"}

    # batched: all queries in one launch per step, autotuned on them
    bcfg, tune_ms = g.autotune_batch(plans, stream)
    b_ms, b_scans = [], None
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b = g.eval_batch(plans, stream, config=bcfg)
        b.rows()
        if i >= args.warmup:
            b_ms.append(1000 * (time.perf_counter() - t0))
            b_scans = b.scans()
        b.close()
    b_q, _ = aggregate_rate(float(np.sum(b_ms)), len(qs) * args.steps, ws, dist)

    # served: Poisson arrivals; the top rate is the headline, K steps of
    # PER_STEP arrivals (fewer when the batched capacity says the run would
    # pass about 90 s; the line then states its arrivals_per_step)
    cap_qps = max(b_q, plain_q)
    per_step = int(min(PER_STEP, max(16, 90.0 * cap_qps / max(1, args.steps + args.warmup))))
    rates = [200, 2000, TOP_RATE]
    served = []
    peaks, which = _peaks()
    srv_cfg = dict(batch=bcfg)
    for rate in rates[:-1]:
        n = int(min(max(100, rate), max(50, 20.0 * cap_qps)))
        sched = np.cumsum(np.random.default_rng(5000 + rate).exponential(1.0 / rate, n))
        srv = gs.Server(g, **srv_cfg)
        lat_us, done_s = srv.replay(plans, sched)
        served.append(_served_entry(srv, rate, n, sched, lat_us, done_s))
        srv.stop()
    top = rates[-1]
    srv = gs.Server(g, **srv_cfg)
    warm = np.cumsum(np.random.default_rng(6000).exponential(1.0 / top, per_step * args.warmup))
    srv.replay(plans, warm)
    n = per_step * args.steps
    sched = np.cumsum(np.random.default_rng(6001).exponential(1.0 / top, n))
    l0 = srv.work()[0]
    barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        lat_us, done_s = srv.replay(plans, sched)
        torch.cuda.synchronize()
    barrier()
    launches = srv.work()[0] - l0
    head = _served_entry(srv, top, n, sched, lat_us, done_s)
    served.append(head)
    srv.stop()
    span_ms = 1000.0 * float(done_s.max() - sched[0])
    value, t_ms = aggregate_rate(span_ms, n, ws, dist)

    # end to end: the same replay with every answer fetched into pinned host memory
    k = max(pl.n_vars for pl in plans)
    pin = torch.empty(max(rows) * k + 16, dtype=torch.int32, pin_memory=True).numpy()
    srv = gs.Server(g, **srv_cfg)
    srv.replay(plans, warm[:per_step], fetch_into=pin)
    lat_e, done_e, fetched = srv.replay(plans, sched, fetch_into=pin)
    srv.stop()
    e2e_value, _ = aggregate_rate(1000.0 * float(done_e.max() - sched[0]), n, ws, dist)
    h2d = int(sum(qs[i % len(qs)].patterns.nbytes for i in range(per_step)))

    # the triple scan over the whole matrix (the bandwidth kernel)
    roof = _scan_roofline(g, w, stream, peaks, which)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = _cpu_baseline(w, triples, qs, args.cpu_seconds)
    if rank == 0:
        print(json.dumps({
            "metric": BANDWIDTH_METRIC,
            "value": value, "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": dict(_bandwidth_config(w, M, len(qs), ws), arrivals_per_step=per_step),
            "setup_s": setup_s,
            "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"],
            "served": served,
            "plain": {"value": plain_q, "unit": "queries/s",
                      "p50_ms": float(np.percentile(lat_ms, 50)),
                      "p99_ms": float(np.percentile(lat_ms, 99)),
                      "timing": "CUDA events around each pass of the queries, one at a time",
                      "phases": phase_summary},
            "batched": {"value": b_q, "unit": "queries/s", "ms_per_step": float(np.mean(b_ms)),
                        "config": bcfg.as_dict(), "autotune_best_ms": tune_ms,
                        "triple_scans_per_step": b_scans[0], "scan_plans_per_step": b_scans[1],
                        "timing": "host wall clock per batch (plan + launch + counts)"},
            "answer_rows": rows,
            "e2e": {"value": e2e_value, "unit": "queries/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": int(fetched // max(1, args.steps)),
                    "path": "gs_server_replay with every answer copied to pinned host memory"},
            "roofline": roof, "cpu_baseline": cpu, "clocks": clk.summary(),
            "gpu_launches": launches,
        }), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _served_entry(srv, rate, n, sched, lat_us, done_s):
    completed, batches, peak = srv.stats()
    launches, scans, scan_plans = srv.work()
    span = float(done_s.max() - sched[0])
    return {"offered_qps": rate, "queries": n, "achieved_qps": n / span,
            "p50_ms": float(np.percentile(lat_us, 50) / 1e3),
            "p99_ms": float(np.percentile(lat_us, 99) / 1e3),
            "batches": batches, "queries_per_batch": n / max(1, batches),
            "triple_scans": scans, "plans_per_scan": scan_plans / max(1, scans),
            "peak_admitted_bytes": peak}


NOMINAL_HBM_GBS = 7700.0   # the B300's nominal HBM3e bandwidth, reported beside the measured peak


def _scan_roofline(g, w, stream, peaks, which, n_scan=20):
    """The triple-scan call (Eq. 17 / Eq. 21 over the whole matrix) timed
    alone with CUDA events: algorithmic bytes 2 (4 (N + 1) + 4 M) + N / 8."""
    import torch
    preds, dirs = [1, 2, 3, 1, 2], [0, 0, 0, 1, 1]
    words = (w.n_vertices + 31) // 32
    out = torch.empty(words, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        g.scan(preds, dirs, out=out)
    se0, se1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(n_scan):
        flush.fill_(1)
        # ~2 ms on the device: the host enqueues the scan meanwhile, so no
        # host delay falls between the two events
        torch.cuda._sleep(4000000)
        se0.record(stream)
        g.scan(preds, dirs, out=out)
        se1.record(stream)
        torch.cuda.synchronize()
        ms.append(se0.elapsed_time(se1))
    g.scan_status()
    scan_ms = float(np.mean(ms))
    N, M = w.n_vertices, g.n_triples
    alg = 2 * (4 * (N + 1) + 4 * M) + N // 8
    achieved = alg / (scan_ms / 1000.0) / 1e9
    return {"kernel": "triple-scan call (gs_scan_candidates: k_scan_zero + k_scan over both "
                      "orientations + k_scan_eval)",
            "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "peak_source": which,
            "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
            "traffic": _scan_traffic(w.name), "algorithmic_bytes": alg, "ms_per_launch": scan_ms,
            "ms_median": float(np.median(ms))}


def run_lspm(args):
    """Per-query LSpMs (Sec. 6.2): for each query of the workload (the
    bandwidth family on rmat26 and with --family bandwidth), the store
    reduced on the device to the predicates its evaluation reads, its size,
    the device time of the reduction, and the query's device time on it
    against the full store (one line; answers checked equal)."""
    import torch
    torch.cuda.set_device(0)
    import paper_2106_14038_b300 as gs
    w, triples, qs = _workload(args.workload, args.family)
    g = gs.Graph(*triples, w.n_vertices, w.n_preds)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = []
    for i, q in enumerate(qs):
        plan = g.plan(q.patterns)
        full_ms, red_ms, build_ms, rows = [], [], [], None
        for rep in range(args.warmup + args.steps):
            r = g.eval(plan, stream)
            n_full = r.info()[0]
            ms_full = r.stats()[0]
            r.close()
            torch.cuda.synchronize()
            e0.record(stream)
            lspm = gs.Lspm.for_plan(g, plan, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            r = lspm.eval(plan, stream)
            n_red = r.info()[0]
            ms_red = r.stats()[0]
            r.close()
            assert n_red == n_full, (i, n_red, n_full)
            if rep >= args.warmup:
                full_ms.append(ms_full)
                red_ms.append(ms_red)
                build_ms.append(e0.elapsed_time(e1))
                rows = n_full
                kept = (lspm.info(False), lspm.info(True))
            lspm.close()
        plan.close()
        out.append({"index": i, "shape": q.shape, "rows": rows,
                    "kept_rows_entries": kept[0], "kept_cols_entries": kept[1],
                    "kept_share": (kept[0][1] + kept[1][1]) / (2.0 * g.n_triples),
                    "full_ms": float(np.median(full_ms)), "lspm_eval_ms": float(np.median(red_ms)),
                    "lspm_build_ms": float(np.median(build_ms))})
    print(json.dumps({
        "metric": "per-query LSpM: device ms of the reduction and of the query on it vs the full store",
        "unit": "ms", "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
        "data": "synthetic", "config": {"workload": w.name, "family": args.family,
                                        "triples": g.n_triples, "queries": len(qs)},
        "queries": out}), flush=True)


def run_paths(args):
    """Per-path binding trees (GS_PLAN_PATHS: one tree per path, tree-pruning,
    join) against the path-linearized tree on the workload's stars,
    snowflakes and cycles, both on the grid path: binding-tree nodes (the
    memory the trees take), answer rows (equal) and device time."""
    import torch
    torch.cuda.set_device(0)
    os.environ["GS_EXEC"] = "grid"          # tree sizes are kept on the grid path
    import paper_2106_14038_b300 as gs
    w, triples, qs = _workload(args.workload)
    g = gs.Graph(*triples, w.n_vertices, w.n_preds)
    stream = torch.cuda.current_stream()
    out = []
    for i, q in enumerate(qs):
        if not q.shape.startswith(("star", "snowflake", "cycle")):
            continue
        row = {"index": i, "shape": q.shape}
        for name, flags in (("linear", gs.PLAN_DEGREE), ("paths", gs.PLAN_PATHS)):
            plan = g.plan(q.patterns, flags)
            ms = []
            for rep in range(args.warmup + args.steps):
                r = g.eval(plan, stream)
                n, _ = r.info()
                if rep >= args.warmup:
                    ms.append(r.stats()[0])
                tree = r.tree()
                r.close()
            row[name] = {"rows": n, "tree_nodes": int(sum(tree)), "per_tree": tree,
                         "device_ms": float(np.mean(ms))}
            plan.close()
        assert row["linear"]["rows"] == row["paths"]["rows"], row
        out.append(row)
    print(json.dumps({"metric": "binding-tree nodes and device ms, per-path vs linearized",
                      "config": {"workload": w.name}, "queries": out}), flush=True)


def main():
    args = _args()
    if args.mode == "paths":
        run_paths(args)
        return
    if args.mode == "lspm" and args.impl == "gsmart":
        run_lspm(args)
        return
    if args.impl == "gsmart" and args.mode == "plain" and args.workload == "rmat26":
        run_bandwidth(args)
        return
    if args.mode == "query" and args.impl == "gsmart":
        run_query(args)
        return
    if args.mode == "scan" and args.impl == "gsmart":
        run_scan_only(args)
        return
    if args.mode == "batched" and args.impl == "gsmart":
        run_batched(args)
        return
    if args.mode == "served" and args.impl == "gsmart":
        run_served(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gsmart(args)


if __name__ == "__main__":
    main()
