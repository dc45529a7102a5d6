"""Benchmark: segmented PageRank (CSR segmenting + frequency-based clustering)
on a directed RMAT scale-25 graph, GTEPS per iteration, against the plain
pull kernel on the same GPU and the FP64 oracle on the host cores.

One step = one PageRank solve: r_0 = 1/V then 20 iterations (damping 0.85),
every iteration one segment-processing gather (Algorithm 3) and one fused
merge + vertex update (Algorithms 4, 5).  value = E * 20 * steps / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--scale S] [--k K] [--sweep]

With torchrun (N > 1) every rank runs an independent replica of the whole
workload on its own GPU (PageRank on one graph is not sharded here); value
sums the replicas' edges over the slowest rank's time.
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

METRIC = "PageRank GTEPS & HBM-roofline %, segmented vs plain pull at ≤1e-5 L1 err"
ITERS = 20
DAMPING = 0.85


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, pg) -> float:
    """The largest x over the process group's ranks (x itself without one)."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: float, world: int, t_max: float) -> float:
    """Whole-job throughput of `world` replicas: all ranks' units over the
    slowest rank's time."""
    return units_per_rank * world / t_max


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def gather_peaks(probes, row_bytes_and_tables, smem=False):
    """Random-read ceilings of this GPU, measured now by the probe library (the
    row gathers are bound by these, not by a streaming copy): {(row_bytes,
    table_bytes): GB/s}, plus shared-memory lookups in G/s when smem."""
    out = {}
    for rb, tb in row_bytes_and_tables:
        out[(rb, tb)] = probes.measure_row_gather(rb, tb) / 1e9
    if smem:
        out["smem"] = probes.measure_smem_lookups() / 1e9
    return out


def _probes():
    from paper_1608_01362_gb300 import probes
    return probes


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


KERNEL_SOURCES = ("seg_gather.cu", "seg_gather.cuh", "pagerank.cu", "update.cuh", "gather.cuh")


def kernel_source_hash():
    """Hash of the sources of the kernels one iteration launches."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1608_01362_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_per_iteration(E, scale=25, segments=None):
    """DRAM bytes per iteration from the committed ncu summary of the RMAT-25
    workload (per edge, scaled to E), when it was taken on the current kernel
    sources, the run is that workload and it runs the profiled plan (the same
    segment count); else None."""
    if scale != 25:
        return None
    try:
        with open(os.path.join(ROOT, "profiles", "pagerank_iteration_rmat25_traffic.json")) as f:
            t = json.load(f)
        if t.get("kernel_source_sha") != kernel_source_hash():
            return None
        if segments is not None and int(t["plan"]["segments"]) != int(segments):
            return None
        return float(t["dram_bytes_per_edge"]) * E
    except Exception:
        return None


def make_graph(scale):
    import graphgen
    t = time.time()
    g = graphgen.rmat(scale, 16, seed=1)
    return g, time.time() - t


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_solution(g):
    """The FP64 oracle on the full graph: 20 plain-pull iterations from
    r_0 = 1/V, with the per-vertex bound on the rounding error of any FP32
    evaluation of them.  Each plain iteration is timed alone (the out-degree
    pass, the allocations and the bound's own work are outside its timer).
    Returns (rank, bound, seconds per iteration, wall seconds of the call)."""
    import oracle
    secs = np.zeros(ITERS)
    t0 = time.time()
    want, bound = oracle.pagerank_bound(g.offsets, g.src, iters=ITERS, iter_seconds=secs)
    return want, bound, secs, time.time() - t0


def cpu_baseline_from(g, secs):
    """cpu_baseline record of the oracle's timed iterations."""
    import oracle
    t = float(np.median(secs))
    return {"value": g.E / t / 1e9, "unit": "GTEPS", "cores": oracle.num_threads(),
            "cpu": cpu_model(), "kind": "oracle",
            "sample": f"{len(secs)} FP64 plain-pull iterations over the full graph "
                      f"(V={g.V}, E={g.E}), each timed alone (set-up excluded); "
                      f"value = E / median iteration time",
            "seconds_per_iteration_median": t}


def parity_report(got, want, bound, tol_l1=1e-5):
    """Element-by-element comparison of an FP32 rank vector with the FP64
    oracle: relative L1 (the metric's gate), the largest error as a fraction
    of its vertex's rounding bound, vertices outside their bound, and the
    largest relative error."""
    err = np.abs(np.asarray(got, np.float64) - want)
    rl1 = float(err.sum() / np.abs(want).sum())
    outside = int(np.count_nonzero(~(err <= bound)))
    return {"rel_l1": rl1, "tol_rel_l1": tol_l1,
            "max_err_over_bound": float(np.max(err / bound)),
            "vertices_outside_bound": outside,
            "max_rel_err": float(np.max(err / want)),
            "ok": bool(rl1 <= tol_l1 and outside == 0)}


def run_reference(args):
    """--impl reference: the FP64 oracle timed on the host cores (rank 0).
    One step = one plain-pull iteration over the full graph, timed inside the
    oracle (set-up excluded, the same routine as the cpu_baseline leg)."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle
    g, _ = make_graph(args.scale)
    n = args.warmup + args.steps
    secs = np.zeros(n)
    oracle.pagerank(g.offsets, g.src, iters=n, iter_seconds=secs)
    dt = float(secs[args.warmup:].sum())
    v = g.E * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GTEPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"pagerank_rmat{args.scale}_directed_ef16", "V": g.V, "E": g.E,
                   "iterations_per_step": 1, "l2_policy": "inputs larger than L2"},
        "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": oracle.num_threads(),
                         "cpu": cpu_model(), "kind": "oracle",
                         "sample": "one FP64 plain-pull iteration per step over the full graph, "
                                   "timed inside the oracle (set-up excluded)"},
        "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_lp(args):
    """Label propagation on an undirected RMAT graph (default scale 24):
    synchronous min-label passes until no label changes, GTEPS per pass."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1608_01362_gb300 import cagra as C
    from paper_1608_01362_gb300 import pipeline as P
    scale = args.scale if args.scale != 25 else 24
    import graphgen
    t = time.time()
    g = graphgen.rmat(scale, 16, seed=1, symmetric=True)
    gen_s = time.time() - t
    graph = P.Graph(g.offsets, g.src, cluster_mode=0)
    bounds = P.plan_bounds(graph, 1, args.plan or 24.0)
    lp = P.LabelPropagation(graph, bounds=bounds, overlap=args.overlap)
    for _ in range(args.warmup):
        lp.run(max_passes=2)
    torch.cuda.synchronize()
    lab = lp.init()
    a, b = lp.labels[0], lp.labels[1]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    changes = []
    start.record()
    while True:  # until a pass changes nothing (each pass reads its count)
        changes.append(C.lp_iterate(lp.seg, a, b))
        a, b = b, a
        if changes[-1] == 0 or len(changes) > 10000:
            break
    stop.record()
    torch.cuda.synchronize()
    dt = start.elapsed_time(stop) / 1e3
    passes = len(changes)
    labels = graph.to_original(a).cpu().numpy()
    line = {"metric": "label propagation GTEPS per pass", "value": g.E * passes / dt / 1e9,
            "unit": "GTEPS", "n_gpus": 1, "steps": passes, "warmup": args.warmup,
            "ms_per_step": dt / passes * 1e3, "higher_is_better": True, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": f"lp_rmat{scale}_undirected_ef16", "V": g.V, "E": g.E,
                       "segments": lp.seg.info["num_segments"], "q": lp.seg.info["q"],
                       "staged_segments": lp.seg.info["staged_segments"]},
            "passes": passes, "components": int(np.unique(labels).size),
            "generate_host_s": gen_s}
    # roofline of one pass: B_min = 4E (arcs) + 8V (offsets) + 12V (labels gathered once,
    # read by the update, written)
    peak, peak_kind = _peaks()
    bmin = 4 * g.E + 20 * g.V
    ach = bmin / (dt / passes) / 1e9
    line["roofline"] = {"bound": "hbm", "kernel": "one pass (gather + merge/update launches)",
                        "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                        "traffic": None, "peak_source": peak_kind, "algorithmic_bytes": bmin}
    line["gpu_launches"] = 4 * passes
    # end to end through the public API: the initial labels from pinned host
    # memory, lp_run to convergence, the final labels back to pinned memory
    init_h = lp.init().cpu().pin_memory()
    out_h = torch.empty_like(init_h).pin_memory()
    torch.cuda.synchronize()
    start.record()
    lp.labels[0].copy_(init_h, non_blocking=True)
    p_e2e, _ = C.lp_run(lp.seg, lp.labels[0])
    out_h.copy_(lp.labels[0], non_blocking=True)
    stop.record()
    stop.synchronize()
    dt_e2e = start.elapsed_time(stop) / 1e3
    line["e2e"] = {"value": g.E * p_e2e / dt_e2e / 1e9, "unit": "GTEPS",
                   "h2d_bytes_per_step": 4 * g.V // max(1, p_e2e),
                   "d2h_bytes_per_step": 4 * g.V // max(1, p_e2e), "passes": int(p_e2e),
                   "result_ok": bool(np.array_equal(graph.to_original(out_h.cuda()).cpu().numpy(),
                                                    labels))}
    if not args.no_cpu_baseline:
        import oracle
        t0 = time.time()
        oracle.label_propagation(g.offsets, g.src, np.arange(g.V, dtype=np.int32), max_passes=1)
        t1 = time.time() - t0
        line["cpu_baseline"] = {"value": g.E / t1 / 1e9, "unit": "GTEPS",
                                "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": "one synchronous pass over the full graph"}
    print(json.dumps(line), flush=True)


def run_batched(args):
    """1,024 independent directed RMAT graphs (scales uniform in 8..15, edge
    factor 16), 20 PageRank iterations each: one persistent launch (captured
    in a CUDA graph) against one segmented handle and pr_iterate per graph."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import graphgen
    from paper_1608_01362_gb300 import cagra as C
    from paper_1608_01362_gb300 import pipeline as P
    t = time.time()
    gs = graphgen.small_graph_batch(count=args.graphs, seed=1, scale_lo=8, scale_hi=15)
    gen_s = time.time() - t
    Etot = sum(len(g.src) for g in gs)
    Vtot = sum(len(g.offsets) - 1 for g in gs)
    # autotune the block size of the batched launch
    best = None
    tune = {}
    for th in (1024, 512, 256):
        bp = P.BatchedPageRank(gs, threads=th)
        bp.run(ITERS)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(3):
            bp.run(ITERS)
        b.record()
        b.synchronize()
        tune[th] = a.elapsed_time(b) / 3e3
        if best is None or tune[th] < tune[best]:
            best = th
        del bp
    bp = P.BatchedPageRank(gs, threads=best)
    # one CUDA graph holding the whole batched solve
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    cg_graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        bp.run(ITERS)
        torch.cuda.synchronize()
        with torch.cuda.graph(cg_graph, stream=s):
            C.pr_batch_run(bp.batch, ITERS, DAMPING, bp.rank)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(args.warmup):
        cg_graph.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        cg_graph.replay()
    b.record()
    b.synchronize()
    t_batch = a.elapsed_time(b) / 1e3 / args.steps
    rank = bp.rank.cpu().numpy()
    # per-graph launches: one segmented handle per graph, pr_iterate per graph
    handles = []
    for g in gs:
        graph = P.Graph(g.offsets, g.src, cluster_mode=None)
        handles.append(P.SegmentedPageRank(graph, 1))
    for h in handles[:8]:
        h.run(ITERS)
    torch.cuda.synchronize()
    a.record()
    for h in handles:
        h.init()
        h.step(h.rank[0], h.contrib[0], h.rank[1], h.contrib[1], DAMPING, ITERS)
    b.record()
    b.synchronize()
    t_per = a.elapsed_time(b) / 1e3
    # the same per-graph launches replayed from one CUDA graph, so that the
    # comparison is of device work, not of host launch cost
    s2 = torch.cuda.Stream()
    s2.wait_stream(torch.cuda.current_stream())
    g_per = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s2):
        for h in handles[:8]:
            h.run(ITERS)
        torch.cuda.synchronize()
        with torch.cuda.graph(g_per, stream=s2, capture_error_mode="relaxed"):
            for h in handles:
                h.init()
                h.step(h.rank[0], h.contrib[0], h.rank[1], h.contrib[1], DAMPING, ITERS)
    torch.cuda.current_stream().wait_stream(s2)
    g_per.replay()
    torch.cuda.synchronize()
    a.record()
    for _ in range(3):
        g_per.replay()
    b.record()
    b.synchronize()
    t_per_graph = a.elapsed_time(b) / 3e3
    # accuracy against the FP64 oracle on a sample of graphs
    import oracle
    errs = []
    for i in range(0, len(gs), max(1, len(gs) // 64)):
        want, _ = oracle.pagerank(gs[i].offsets, gs[i].src, iters=ITERS)
        got = rank[bp.vbase[i]:bp.vbase[i + 1]].astype(np.float64)
        errs.append(float(np.abs(got - want).sum() / np.abs(want).sum()))
    line = {"metric": "batched PageRank GTEPS (20 iterations per graph)",
            "value": Etot * ITERS / t_batch / 1e9, "unit": "GTEPS", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch * 1e3,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched_pagerank_{len(gs)}_rmat_scales_8_15_ef16",
                       "graphs": len(gs), "V": Vtot, "E": Etot, "threads": best,
                       "cuda_graph": True},
            "autotune_ms": {str(k): v * 1e3 for k, v in tune.items()},
            "per_graph_launches_ms": t_per * 1e3, "speedup_vs_per_graph": t_per / t_batch,
            "per_graph_launches_cuda_graph_ms": t_per_graph * 1e3,
            "speedup_vs_per_graph_cuda_graph": t_per_graph / t_batch,
            "max_rel_l1_vs_oracle": max(errs), "oracle_sample_graphs": len(errs),
            "generate_host_s": gen_s}
    # roofline of one solve of all graphs: the method needs the edges and the
    # per-vertex arrays from HBM once (a graph's iterations run on chip, its
    # edges re-read from L2): B_min = 4E + 8(V + G) offsets + 4V degrees + 4V ranks
    peak, peak_kind = _peaks()
    bmin = 4 * Etot + 8 * (Vtot + len(gs)) + 8 * Vtot
    ach = bmin / t_batch / 1e9
    line["roofline"] = {"bound": "hbm", "kernel": "batch_pagerank_kernel (one solve, 20 iterations)",
                        "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                        "traffic": None, "peak_source": peak_kind, "algorithmic_bytes": bmin,
                        "note": "iterations 2-20 re-read each graph's edges from L2, so the "
                                "solve is bound by L2 and latency, not HBM"}
    line["gpu_launches"] = args.steps
    # end to end: the solve through the public call (pr_batch_run) with every
    # graph's ranks read back into pinned host memory
    rank_h = torch.empty(bp.rank.numel(), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    a.record()
    for _ in range(args.steps):
        C.pr_batch_run(bp.batch, ITERS, DAMPING, bp.rank)
        rank_h.copy_(bp.rank, non_blocking=True)
    b.record()
    b.synchronize()
    t_e2e = a.elapsed_time(b) / 1e3 / args.steps
    line["e2e"] = {"value": Etot * ITERS / t_e2e / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 4 * int(bp.rank.numel()),
                   "note": "graphs stay resident on the device between solves",
                   "result_ok": bool(np.array_equal(rank_h.numpy(), rank))}
    print(json.dumps(line), flush=True)


def ppr_seeds(g, n=64, seed=1):
    """n distinct seed vertices among those with out-edges, drawn in order from
    SplitMix64 stream (seed, 0) (duplicates skipped)."""
    import graphgen
    cand = np.flatnonzero(np.bincount(g.src, minlength=len(g.offsets) - 1) > 0)
    out = []
    draws = graphgen.splitmix_draws(seed, 0, 64 * n)
    for d in draws:
        v = int(cand[int(d % np.uint64(len(cand)))])
        if v not in out:
            out.append(v)
            if len(out) == n:
                break
    return np.asarray(out, dtype=np.int32)


def _ppr_bounds(nd, V, k):
    """k uniform segments over the sources with out-edges [0, nd) of the
    clustered numbering, and one edgeless segment [nd, V)."""
    b = [int(round(i * nd / k)) for i in range(k + 1)]
    if nd < V:
        b.append(V)
    return np.unique(np.asarray(b, dtype=np.int64))


def run_ppr(args):
    """64 personalised PageRank vectors on a directed RMAT graph (default
    scale 22), 20 iterations, rank matrix stored as BF16 hi+lo planes with
    FP32 accumulation: one batched solve against 64 single-vector solves."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1608_01362_gb300 import cagra as C
    from paper_1608_01362_gb300 import pipeline as P
    scale = args.scale if args.scale != 25 else 22
    g, gen_s = make_graph(scale)
    graph = P.Graph(g.offsets, g.src, cluster_mode=0)
    nd = int((graph.outdeg > 0).sum().item())
    seeds = ppr_seeds(g)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def time_solve(b, reps=2, iters=ITERS):
        b.init(seeds)
        C.ppr_batched_iterate(b.ppr, graph.inv, DAMPING, 2)
        torch.cuda.synchronize()
        a, z = ev(), ev()
        a.record()
        for _ in range(reps):
            C.ppr_batched_iterate(b.ppr, graph.inv, DAMPING, iters)
        z.record()
        z.synchronize()
        return a.elapsed_time(z) / 1e3 / (reps * iters)

    # autotune the segment count (Section III-D's trade-off, 64-wide rows)
    tune = {}
    best = None
    for planes in (2, 1):
        for k in (args.k,) if args.k else (1, 2, 4, 8, 16, 32):
            b = P.BatchedPPR(graph, bounds=_ppr_bounds(nd, graph.V, k), planes=planes)
            t = time_solve(b, reps=1, iters=5)
            tune[f"planes{planes}_k{k}"] = {"ms_per_iter": t * 1e3, "q": b.seg.info["q"],
                                            "bytes": b.ppr.bytes}
            if planes == 2 and (best is None or t < tune[f"planes2_k{best}"]["ms_per_iter"] / 1e3):
                best = k
            del b
    # the dense hub block on the tensor cores: its size (0: none)
    best_h = args.dense if args.dense >= 0 else None
    if best_h is None:
        for hh in (0, 4096, 8192, 16384, 32768):
            b = P.BatchedPPR(graph, bounds=_ppr_bounds(nd, graph.V, best), planes=2,
                             dense_hubs=hh)
            t = time_solve(b, reps=1, iters=5)
            tune[f"dense_h{hh}"] = {"ms_per_iter": t * 1e3, "q": b.seg.info["q"]}
            if best_h is None or t < tune[f"dense_h{best_h}"]["ms_per_iter"] / 1e3:
                best_h = hh
            del b
    b = P.BatchedPPR(graph, bounds=_ppr_bounds(nd, graph.V, best), planes=2, dense_hubs=best_h)
    info = b.seg.info
    # timed: steps x (init + 20 iterations), inputs resident in HBM (the
    # 1 GB rank matrix and 0.5 GB BF16 planes exceed L2: no flush needed)
    for _ in range(args.warmup):
        b.init(seeds)
        C.ppr_batched_iterate(b.ppr, graph.inv, DAMPING, ITERS, b.rank)
    torch.cuda.synchronize()
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    a, z = ev(), ev()
    a.record()
    for _ in range(args.steps):
        b.init(seeds)
        C.ppr_batched_iterate(b.ppr, graph.inv, DAMPING, ITERS, b.rank)
    z.record()
    z.synchronize()
    clocks = clk.stop()
    t_step = a.elapsed_time(z) / 1e3 / args.steps
    # per launch of one iteration
    phase_ms = {}
    for ph, name in ((1, "gather"), (8, "dense_tensor_core"), (2, "fixup"), (4, "merge")):
        if ph == 8 and not best_h:
            continue
        b.init(seeds)
        C.ppr_batched_iterate(b.ppr, graph.inv, DAMPING, 2)
        ts = []
        for _ in range(5):
            C.ppr_batched_step(b.ppr, graph.inv, DAMPING, 15 - ph)  # the others, untimed
            e0, e1 = ev(), ev()
            e0.record()
            C.ppr_batched_step(b.ppr, graph.inv, DAMPING, ph)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        phase_ms[name] = float(np.median(ts))
    # result in original IDs, errors against the oracle on sampled columns
    b.init(seeds)
    R, resid = b.run(seeds, ITERS)
    Rh = R.cpu().numpy()
    import oracle
    cols = np.array([0, 21, 42, 63])
    t0 = time.time()
    want = oracle.ppr(g.offsets, g.src, seeds[cols], iters=ITERS)
    oracle_s = time.time() - t0
    err = np.abs(Rh[:, cols].astype(np.float64) - want).sum(0) / np.abs(want).sum(0)
    # per entry: the FP64 rounding bound (accumulation 2^-23 when the tensor
    # cores add the hub block: a truncating FP32 sum at most doubles each
    # addition's relative error)
    u_acc = 2.0 ** -23 if best_h else oracle.U_FP32
    worst, outside = 0.0, 0
    for j, c in enumerate(cols):
        _, bnd = oracle.pagerank_bound(g.offsets, g.src, iters=ITERS, seed=int(seeds[c]),
                                       u_acc=u_acc, u_store=oracle.U_BF16X2)
        e = np.abs(Rh[:, c].astype(np.float64) - want[:, j])
        m = bnd > 0
        worst = max(worst, float(np.max(e[m] / bnd[m])))
        outside += int(np.count_nonzero(e > bnd))
    dense_rec = None
    if best_h:
        # 64-source chunks with an edge in each 128-destination tile (the MMAs issued)
        hb = b.bits.reshape(best_h // 128, 128, best_h // 64, 2)
        nz_chunks = int((hb != 0).any(dim=3).any(dim=1).sum().item())
        flops = nz_chunks * 128 * 64 * 64 * 2 * 2
        t_d = phase_ms["dense_tensor_core"] / 1e3
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                bf16_peak, bf16_kind = float(json.load(f)["bf16_tflops"]), "measured"
        except Exception:
            bf16_peak, bf16_kind = 1900.0, "fallback"
        dense_rec = {"hubs": best_h, "hub_block_edges": int(g.E - b.rest_src.numel()),
                     "hub_block_edge_share": float((g.E - b.rest_src.numel()) / g.E),
                     "tile_chunks": nz_chunks, "mma_flops": flops,
                     "tflops": flops / t_d / 1e12, "bf16_peak_tflops": bf16_peak,
                     "peak_kind": bf16_kind, "frac": flops / t_d / 1e12 / bf16_peak,
                     "ms": t_d * 1e3}
    # 64 single-vector solves through the segmented PageRank path
    cand, _ = P.autotune_segments(graph)
    sp = P.build_candidate(graph, cand)
    r1, _ = sp.run_ppr(int(seeds[0]), ITERS)
    err1 = float(np.abs(r1.cpu().numpy() - want[:, 0]).sum() / np.abs(want[:, 0]).sum())
    torch.cuda.synchronize()
    a.record()
    for s in seeds:
        sp.run_ppr(int(s), ITERS)
    z.record()
    z.synchronize()
    t_single = a.elapsed_time(z) / 1e3
    # end to end through the public API: seeds in from the host, R out to pinned host memory
    Rhost = torch.empty_like(b.rank, device="cpu").pin_memory()
    torch.cuda.synchronize()
    a.record()
    for _ in range(max(1, args.steps // 2)):
        b.run(seeds, ITERS)
        Rhost.copy_(b.rank, non_blocking=True)
    z.record()
    z.synchronize()
    t_e2e = a.elapsed_time(z) / 1e3 / max(1, args.steps // 2)
    # roofline of the dominant launch (algorithmic bytes per launch)
    pl = 2
    cbytes = 128 * pl * nd
    rows = int(info["rows"])
    alg = {"gather": 4 * g.E + cbytes + 256 * rows + 8 * b.ppr.chunks,
           "fixup": 0, "merge": 256 * rows + 4 * rows + 8 * graph.V + cbytes}
    dom = max(("gather", "merge"), key=lambda n: phase_ms[n])
    peak, peak_kind = _peaks()
    ach = alg[dom] / (phase_ms[dom] / 1e3) / 1e9
    edge_cols = g.E * 64 * ITERS
    # the gather reads one 64-column row (BF16 hi+lo: 256 bytes) per edge from a
    # table of the non-dangling sources' rows; its ceiling is the random-row
    # rate of such a table (measured now); hub rows reread from L1/L2 can
    # carry it above that rate
    rb = 128 * pl
    gp = gather_peaks(_probes(), [(rb, rb * nd)])
    a_rows = g.E * rb / (phase_ms["gather"] / 1e3) / 1e9
    gather_rows = {"bound": "random rows", "unit": "GB/s", "row_bytes": rb,
                   "table_bytes": rb * nd, "achieved": a_rows, "peak": gp[(rb, rb * nd)],
                   "frac": a_rows / gp[(rb, rb * nd)]}
    line = {"metric": "batched personalised PageRank: edge-vector GTEPS (64 vectors x 20 "
                      "iterations) at BF16 hi+lo storage",
            "value": edge_cols / t_step / 1e9, "unit": "GTEPS (edge x vector)", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
            "higher_is_better": True, "dtype": "bf16x2 storage, f32 accumulate",
            "data": "synthetic",
            "config": {"workload": f"ppr64_rmat{scale}_ef16", "V": g.V, "E": g.E,
                       "nondangling": nd, "segments": info["num_segments"], "q": info["q"],
                       "planes": 2, "dense_hubs": best_h, "l2_flush": "inputs larger than L2"},
            "vs_baseline": None,
            "kernels_ms_per_iteration": phase_ms,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak,
                         "unit": "GB/s", "frac": ach / peak, "traffic": None,
                         "peak_source": peak_kind, "algorithmic_bytes": alg[dom]},
            "gather_row_bound": gather_rows,
            "single_vector_64_runs_ms": t_single * 1e3,
            "speedup_vs_64_single_runs": t_single / t_step,
            "rel_l1_vs_oracle_sampled_columns": {int(c): float(e) for c, e in zip(cols, err)},
            "sampled_columns_max_err_over_bound": worst,
            "sampled_columns_entries_outside_bound": outside,
            "dense_hub_block": dense_rec,
            "single_vector_rel_l1_col0": err1,
            "autotune": tune, "clocks": clocks,
            "e2e": {"value": edge_cols / t_e2e / 1e9, "unit": "GTEPS (edge x vector)",
                    "h2d_bytes_per_step": 64 * 4, "d2h_bytes_per_step": int(Rhost.numel() * 4)},
            "gpu_launches": args.steps * (3 * ITERS + 1),
            "generate_host_s": gen_s, "oracle_4_columns_s": oracle_s}
    if not args.no_cpu_baseline:
        t0 = time.time()
        oracle.ppr(g.offsets, g.src, seeds, iters=1)
        t1 = time.time() - t0
        line["cpu_baseline"] = {"value": g.E * 64 / t1 / 1e9, "unit": "GTEPS (edge x vector)",
                                "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": "one iteration of all 64 vectors over the full graph"}
    print(json.dumps(line), flush=True)


def run_cf(args):
    """Collaborative filtering on the Netflix-shaped bipartite graph (480,189
    users x 17,770 items x 99M ratings), K = 32, lambda 0.05, step 1e-3, 10
    sweeps, factors stored in FP32, BF16 and BF16 hi+lo; RMSE per sweep
    against the FP64 oracle on the same inputs."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import graphgen
    import oracle
    from paper_1608_01362_gb300 import cagra as C
    K, LAM, STEP, SWEEPS = 32, 0.05, 1e-3, 10
    t = time.time()
    bp = graphgen.bipartite(seed=1)
    gen_s = time.time() - t
    U, I, R = bp.U, bp.I, bp.R
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).cuda()  # noqa: E731
    uoff, uitem, urate = dev(bp.user_offsets, torch.int64), dev(bp.items, torch.int32), \
        dev(bp.ratings, torch.uint8)
    ioff = torch.empty(I + 1, dtype=torch.int64, device="cuda")
    iuser = torch.empty(R, dtype=torch.int32, device="cuda")
    irate = torch.empty(R, dtype=torch.uint8, device="cuda")
    C.cf_transpose(U, I, uoff, uitem, urate, ioff, iuser, irate)
    P0, Q0 = graphgen.cf_factors(U, I, K, seed=1)
    P0d, Q0d = dev(P0, torch.float32), dev(Q0, torch.float32)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    res = {}
    for prec, name in ((2, "bf16x2"), (1, "bf16"), (0, "fp32")):
        h = C.cf_create(U, I, K, prec, uoff, uitem, urate, ioff, iuser, irate)
        for _ in range(args.warmup):
            C.cf_set_factors(h, P0d, Q0d)
            C.cf_sweep(h, 1, LAM, STEP)
        sse = torch.zeros(SWEEPS, dtype=torch.float64, device="cuda")
        C.cf_set_factors(h, P0d, Q0d)
        torch.cuda.synchronize()
        clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) if prec == 2 else None
        if clk:
            clk.start()
        a, z = ev(), ev()
        a.record()
        C.cf_sweep(h, SWEEPS, LAM, STEP, sse)
        z.record()
        z.synchronize()
        clocks = clk.stop() if clk else None
        t_sweep = a.elapsed_time(z) / 1e3 / SWEEPS
        phase = {}
        for ph, nm in ((0, "user_gather"), (1, "item_gather"), (2, "user_update"),
                       (3, "item_update")):
            e0, e1 = ev(), ev()
            e0.record()
            C.cf_sweep_phase(h, ph, LAM, STEP)
            e1.record()
            e1.synchronize()
            phase[nm] = e0.elapsed_time(e1)
        res[name] = {"ms_per_sweep": t_sweep * 1e3, "rmse": np.sqrt(sse.cpu().numpy() / R),
                     "kernels_ms": phase, "info": h.info, "clocks": clocks}
        if prec == 2:
            # end to end: factors in from pinned host memory, 10 sweeps, factors out
            Ph = torch.from_numpy(P0.astype(np.float32)).pin_memory()
            Qh = torch.from_numpy(Q0.astype(np.float32)).pin_memory()
            Pd, Qd = torch.empty_like(P0d), torch.empty_like(Q0d)
            torch.cuda.synchronize()
            a.record()
            Pd.copy_(Ph, non_blocking=True)
            Qd.copy_(Qh, non_blocking=True)
            C.cf_set_factors(h, Pd, Qd)
            C.cf_sweep(h, SWEEPS, LAM, STEP)
            C.cf_get_factors(h, Pd, Qd)
            Ph.copy_(Pd, non_blocking=True)
            Qh.copy_(Qd, non_blocking=True)
            z.record()
            z.synchronize()
            res[name]["e2e_s"] = a.elapsed_time(z) / 1e3
        del h
    # FP64 oracle on the same inputs
    t = time.time()
    io, iu, ir = oracle.item_major(U, I, bp.user_offsets, bp.items, bp.ratings)
    P, Q = P0.astype(np.float32).astype(np.float64), Q0.astype(np.float32).astype(np.float64)
    want = []
    t1 = None
    for i in range(SWEEPS):
        t0 = time.time()
        P, Q, e = oracle.cf_sweep(U, I, bp.user_offsets, bp.items, bp.ratings, io, iu, ir, P, Q,
                                  LAM, STEP)
        t1 = t1 or (time.time() - t0)
        want.append(e)
    oracle_s = time.time() - t
    rmse64 = np.sqrt(np.array(want) / R)
    for name in res:
        res[name]["max_abs_rmse_diff_vs_fp64"] = float(np.max(np.abs(res[name]["rmse"] - rmse64)))
        res[name]["final_rmse"] = float(res[name]["rmse"][-1])
        res[name]["rmse"] = [float(x) for x in res[name]["rmse"]]
    head = res["bf16x2"]
    t_sweep = head["ms_per_sweep"] / 1e3
    peak, peak_kind = _peaks()
    # algorithmic DRAM bytes per sweep: both rating CSRs (4 + 1 bytes per
    # rating each), offsets, and each factor row read and written once
    # (BF16 hi+lo: 4 bytes per entry)
    alg = 2 * 5 * R + 8 * (U + I + 2) + 2 * (U + I) * K * 4
    dom = max(head["kernels_ms"], key=head["kernels_ms"].get)
    dom_bytes = 5 * R + (U + I) * K * 4
    ach = dom_bytes / (head["kernels_ms"][dom] / 1e3) / 1e9
    # the gathers read one factor row (4K bytes) per rating at random from an
    # L2-resident table: their ceiling is L2's random-row rate, measured now
    rb = 4 * K
    gp = gather_peaks(_probes(), [(rb, I * rb), (rb, U * rb)])
    gathers_l2 = {}
    for nm, tb in (("user_gather", I * rb), ("item_gather", U * rb)):
        a = R * rb / (head["kernels_ms"][nm] / 1e3) / 1e9
        gathers_l2[nm] = {"bound": "L2 random rows", "unit": "GB/s", "row_bytes": rb,
                          "table_bytes": tb, "achieved": a, "peak": gp[(rb, tb)],
                          "frac": a / gp[(rb, tb)]}
    line = {"metric": "collaborative filtering sweep: ratings x sides per second (GTEPS), K=32, "
                      "BF16 hi+lo storage, RMSE diff vs FP64",
            "value": 2 * R / t_sweep / 1e9, "unit": "GTEPS (rating x side)", "n_gpus": 1,
            "steps": SWEEPS, "warmup": args.warmup, "ms_per_step": t_sweep * 1e3,
            "higher_is_better": True, "dtype": "bf16x2 storage, f32 accumulate",
            "data": "synthetic",
            "config": {"workload": "cf_netflix_shaped_480189x17770_99M_K32", "U": U, "I": I,
                       "R": R, "K": K, "lambda": LAM, "step": STEP, "sweeps": SWEEPS,
                       "l2_flush": "none: factors are L2-resident by design; rating CSRs 1 GB"},
            "vs_baseline": None,
            "precisions": res, "rmse_fp64": [float(x) for x in rmse64],
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak,
                         "unit": "GB/s", "frac": ach / peak, "traffic": None,
                         "peak_source": peak_kind, "algorithmic_bytes": dom_bytes,
                         "note": "gathers are L2-bound: every rating reads a factor row "
                                 "from L2 (factors stay resident)"},
            "gathers_l2_bound": gathers_l2,
            "sweep_algorithmic_dram_bytes": alg,
            "clocks": head["clocks"],
            "e2e": {"value": 2 * R * SWEEPS / head["e2e_s"] / 1e9, "unit": "GTEPS (rating x side)",
                    "h2d_bytes_per_step": (U + I) * K * 4 // SWEEPS,
                    "d2h_bytes_per_step": (U + I) * K * 4 // SWEEPS},
            "gpu_launches": 4 * SWEEPS, "generate_host_s": gen_s, "oracle_10_sweeps_s": oracle_s}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = {"value": 2 * R / t1 / 1e9, "unit": "GTEPS (rating x side)",
                                "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": "one FP64 sweep over the full rating graph"}
    print(json.dumps(line), flush=True)


ORDERS = ("generator", "random", "clustered_outdeg", "clustered_threshold")


def _order_graph(P, gens, order, dev="cuda"):
    """The RMAT graph in one vertex order: the generator's own IDs (hubs at
    low IDs: locality), the benchmark's randomly permuted IDs, or that graph
    renumbered by frequency-based clustering (mode 0: out-degree; mode 1:
    out-degree over the average degree, Section V)."""
    if order == "generator":
        g = gens["generator"]
        return P.Graph(g.offsets, g.src, cluster_mode=None, device=dev)
    g = gens["random"]
    mode = {"random": None, "clustered_outdeg": 0, "clustered_threshold": 1}[order]
    return P.Graph(g.offsets, g.src, cluster_mode=mode, device=dev)


def run_qfactor(args):
    """Expansion factor q(k) = subgraph rows / V (Section III-D, Fig. qfactor)
    of the paper's uniform split into k segments, k = 1..64, in four vertex
    orders, from the GPU segment builder (Algorithm 2)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import graphgen
    from paper_1608_01362_gb300 import cagra as C
    from paper_1608_01362_gb300 import pipeline as P
    t = time.time()
    gens = {"random": graphgen.rmat(args.scale, 16, seed=1),
            "generator": graphgen.rmat(args.scale, 16, seed=1, permute=False)}
    gen_s = time.time() - t
    ks = (1, 2, 4, 8, 16, 32, 64)
    q = {}
    for order in ORDERS:
        graph = _order_graph(P, gens, order)
        q[order] = {}
        for k in ks:
            seg = C.pr_build_segments(graph.offsets, graph.src, k)
            q[order][k] = float(seg.info["q"])
            seg.close()
        del graph
        torch.cuda.empty_cache()
    g = gens["random"]
    ratio = {k: q["random"][k] / q["clustered_outdeg"][k] for k in ks}
    print(json.dumps({
        "metric": "expansion factor q(k) of k uniform segments", "unit": "rows per vertex",
        "config": {"workload": f"qfactor_rmat{args.scale}_directed_ef16", "V": g.V, "E": g.E,
                   "k": list(ks), "orders": list(ORDERS)},
        "q": q, "q_random_over_clustered": ratio, "generate_host_s": gen_s}), flush=True)


def _phase_times(C, pr, graph, iters=ITERS, reps=2):
    """Mean seconds per iteration of the gather launches and of the merge +
    update launch of a segmented PageRank (CUDA events on the stream)."""
    import torch
    stream = torch.cuda.current_stream()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(iters * reps)] for _ in range(3)]
    pr.init()
    rin, cin, rout, cout = pr.rank[0], pr.contrib[0], pr.rank[1], pr.contrib[1]
    for i in range(iters * reps):
        ev[0][i].record(stream)
        C.cg_seg_gather(pr.seg, C.CG_OP_SUM_F32, cin, None)
        ev[1][i].record(stream)
        C.pr_merge_update(pr.seg, graph.inv, rin, rout, cout, DAMPING, pr.dangling, pr.dangling,
                          None)
        ev[2][i].record(stream)
        rin, cin, rout, cout = rout, cout, rin, cin
    torch.cuda.synchronize()
    tg = float(np.mean([a.elapsed_time(b) for a, b in zip(ev[0], ev[1])])) / 1e3
    tm = float(np.mean([a.elapsed_time(b) for a, b in zip(ev[1], ev[2])])) / 1e3
    return tg, tm


def run_sweep(args):
    """Segment-count sweep (the paper's Fig. seg-breakdown): uniform k =
    1..64 in the random (benchmark) order and the clustered order, plus the
    GPU plan, each with its gather / merge split per iteration and GTEPS."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1608_01362_gb300 import cagra as C
    from paper_1608_01362_gb300 import pipeline as P
    g, gen_s = make_graph(args.scale)
    rows = []
    for order, mode in (("random", None), ("clustered_outdeg", 0)):
        graph = P.Graph(g.offsets, g.src, cluster_mode=mode)
        cands = [("uniform", k) for k in (1, 2, 4, 8, 16, 32, 64)]
        if mode is not None:
            cands.append(("plan", args.plan or 32.0))
        for kind, x in cands:
            pr = (P.SegmentedPageRank(graph, x) if kind == "uniform" else
                  P.SegmentedPageRank(graph, bounds=P.plan_bounds(graph, 1, x)))
            tg, tm = _phase_times(C, pr, graph)
            inf = pr.info
            rows.append({"order": order, "kind": kind,
                         ("k" if kind == "uniform" else "min_avg_degree"): x,
                         "segments": inf["num_segments"], "q": round(inf["q"], 4),
                         "staged_segments": inf["staged_segments"],
                         "gather_ms": tg * 1e3, "merge_update_ms": tm * 1e3,
                         "gteps": g.E / (tg + tm) / 1e9})
            pr.seg.close()
            del pr
        del graph
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "PageRank GTEPS per iteration by segment count",
                      "unit": "GTEPS", "config": {"workload": f"sweep_rmat{args.scale}_directed_ef16",
                                                  "V": g.V, "E": g.E},
                      "rows": rows, "generate_host_s": gen_s}), flush=True)


def run_profile(args):
    """One arm alone, for short ncu captures: `--arm plain_random` (plain
    pull, random order), `plain_clustered`, or `segmented` (the GPU plan,
    --plan threshold, clustered), `--iters` iterations after one warm-up."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1608_01362_gb300 import pipeline as P
    g, _ = make_graph(args.scale)
    if args.arm == "plain_random":
        pr = P.PlainPageRank(P.Graph(g.offsets, g.src, cluster_mode=None))
    elif args.arm == "plain_clustered":
        pr = P.PlainPageRank(P.Graph(g.offsets, g.src, cluster_mode=0))
    else:
        graph = P.Graph(g.offsets, g.src, cluster_mode=0)
        pr = P.SegmentedPageRank(graph, bounds=P.plan_bounds(graph, 1, args.plan or 32.0))
    del g
    pr.init()
    pr.step(pr.rank[0], pr.contrib[0], pr.rank[1], pr.contrib[1], DAMPING, 1)
    torch.cuda.synchronize()
    t = P.time_iterations(pr, args.iters)
    print(json.dumps({"arm": args.arm, "scale": args.scale, "ms_per_iteration": t * 1e3}),
          flush=True)


def run_bc(args):
    """Betweenness centrality from 12 sources (the paper's Table V: runtime
    for 12 starting points) on the directed RMAT graph (default scale 25),
    clustered, with the random (benchmark) order beside it; two sources are
    checked against the FP64 oracle (levels and path counts bit for bit,
    dependencies within the FP64 bound)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_1608_01362_gb300 import cagra as C
    from paper_1608_01362_gb300 import pipeline as P
    g, gen_s = make_graph(args.scale)
    S = ppr_seeds(g, n=12)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    res = {}
    for order, mode in (("clustered_outdeg", 0), ("random", None)):
        graph = P.Graph(g.offsets, g.src, cluster_mode=mode)
        t0 = time.time()
        bc = P.Betweenness(graph)
        torch.cuda.synchronize()
        prep = time.time() - t0
        tune = {}
        for alpha in (0.0, 2.0, 4.0, 16.0, 64.0):  # push/pull switch (0: push only), timed on two sources
            C.bc_set_direction(bc.h, alpha)
            bc.run(S[:1])
            a, z = ev(), ev()
            a.record()
            bc.run(S[:2])
            z.record()
            z.synchronize()
            tune[alpha] = a.elapsed_time(z) / 2e3
        alpha = min(tune, key=tune.get)
        C.bc_set_direction(bc.h, alpha)
        for _ in range(args.warmup):
            bc.run(S[:2])
        torch.cuda.synchronize()
        clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) if mode == 0 else None
        if clk:
            clk.start()
        times = []
        for _ in range(max(1, args.steps // 5)):
            a, z = ev(), ev()
            a.record()
            out = bc.run(S)
            z.record()
            z.synchronize()
            times.append(a.elapsed_time(z) / 1e3)
        clocks = clk.stop() if clk else None
        t12 = float(np.median(times))
        info = C.bc_source_state(bc.h)
        res[order] = {"s_for_12_sources": t12, "alpha": alpha, "alpha_tune_s_per_source": tune,
                      "last_source_levels": info["depth"], "push_levels": info["push_levels"],
                      "pull_levels": info["pull_levels"], "prep_s": prep, "clocks": clocks}
        if mode == 0:
            bc_cl = out.cpu().numpy()
            # end to end: sources from the host, the centrality back to the host
            out_h = torch.empty(g.V, dtype=torch.float64).pin_memory()
            a, z = ev(), ev()
            a.record()
            bc.bc.zero_()
            C.bc_run(bc.h, [graph.to_clustered_id(int(x)) for x in S], bc.bc)
            out_h.copy_(bc.to_original8(bc.bc), non_blocking=True)
            z.record()
            z.synchronize()
            res[order]["e2e_s"] = a.elapsed_time(z) / 1e3
            res[order]["e2e_ok"] = bool(np.array_equal(out_h.numpy(), bc_cl))
            # parity: the first two sources against the oracle
            t0 = time.time()
            out_off, out_dst = oracle.out_csr(g.offsets, g.src)
            par = {"sources": [int(x) for x in S[:2]]}
            worst = 0.0
            for x in S[:2]:
                tt = time.time()
                lev, sig, dl, depth = oracle.bc_source(out_off, out_dst, int(x))
                res[order].setdefault("oracle_s_per_source", time.time() - tt)
                bc.run([int(x)])
                glev, gsig, gdl, ginfo = bc.source_state()
                par.setdefault("levels_equal", True)
                par["levels_equal"] &= bool(np.array_equal(glev.cpu().numpy(), lev))
                par.setdefault("sigma_equal", True)
                par["sigma_equal"] &= bool(np.array_equal(gsig.cpu().numpy(), sig))
                tol = 2.0 * depth * (int(np.diff(out_off).max()) + 8) * 2.0 ** -53
                gd = gdl.cpu().numpy()
                m = dl > 0
                worst = max(worst, float(np.max(np.abs(gd[m] - dl[m]) / dl[m])) / tol)
                par.setdefault("zero_delta_equal", True)
                par["zero_delta_equal"] &= bool(np.all(gd[~m] == 0.0))
            par["max_rel_err_over_tol"] = worst
            par["ok"] = bool(par["levels_equal"] and par["sigma_equal"] and worst <= 1.0 and
                             par["zero_delta_equal"])
            par["oracle_wall_s"] = time.time() - t0
            res[order]["parity"] = par
        del bc, graph
        torch.cuda.empty_cache()
    head = res["clustered_outdeg"]
    t12 = head["s_for_12_sources"]
    line = {"metric": "betweenness centrality, 12 sources: traversed edges per second "
                      "(12 x E / time)",
            "value": 12 * g.E / t12 / 1e9, "unit": "GTEPS", "n_gpus": 1, "steps": len(S),
            "warmup": args.warmup, "ms_per_step": t12 / len(S) * 1e3, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"bc_12_sources_rmat{args.scale}_directed_ef16",
                       "V": g.V, "E": g.E, "sources": [int(x) for x in S],
                       "l2_policy": "inputs larger than L2"},
            "vs_baseline": None, "s_for_12_sources": t12,
            "paper_context": "Table V: 7.08 s for 12 sources on RMAT25 (Xeon, 48 threads)",
            "orders": res, "parity": head["parity"],
            "speedup_clustered_vs_random": res["random"]["s_for_12_sources"] / t12,
            "clocks": head["clocks"],
            "e2e": {"value": 12 * g.E / head["e2e_s"] / 1e9, "unit": "GTEPS",
                    "h2d_bytes_per_step": 4, "d2h_bytes_per_step": 8 * g.V // 12,
                    "result_ok": head["e2e_ok"]},
            "generate_host_s": gen_s}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = {"value": g.E / head["oracle_s_per_source"] / 1e9, "unit": "GTEPS",
                                "cores": 1, "cpu": cpu_model(), "kind": "oracle",
                                "sample": "one source (BFS + dependency pass) over the full "
                                          "graph, single-threaded FP64 Brandes"}
    print(json.dumps(line), flush=True)


def extras(g25, graph25):
    """Compact records of the other forms of the gather, attached to the
    default line so that one run measures them all: label propagation
    (RMAT-24 undirected), 64-vector personalised PageRank (RMAT-22), the
    1,024-graph batch, collaborative filtering (Netflix-shaped) and
    betweenness centrality (RMAT-25, 12 sources).  Each is timed with CUDA
    events and checked against the FP64 oracle on a bounded sample (BC:
    against itself across directions; its oracle runs in the tests)."""
    import torch
    import graphgen
    import oracle
    from paper_1608_01362_gb300 import cagra as C
    from paper_1608_01362_gb300 import pipeline as P
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    out = {}

    def timed(fn, reps=1):
        a, z = ev(), ev()
        a.record()
        for _ in range(reps):
            fn()
        z.record()
        z.synchronize()
        return a.elapsed_time(z) / 1e3 / reps

    # label propagation: passes until no label changes; the first pass bit for bit
    t0 = time.time()
    g = graphgen.rmat(24, 16, seed=1, symmetric=True)
    graph = P.Graph(g.offsets, g.src, cluster_mode=0)
    lp = P.LabelPropagation(graph, bounds=P.plan_bounds(graph, 1, 24.0))
    lp.run(max_passes=2)
    lab = lp.init()
    a_, b_ = lp.labels[0], lp.labels[1]
    C.lp_iterate(lp.seg, a_, b_)
    first = graph.to_original(b_).cpu().numpy()
    want1, _ = oracle.label_propagation_pass(g.offsets, g.src, np.arange(g.V, dtype=np.int32))
    lp.init()
    st, sp = ev(), ev()
    st.record()
    passes = 0
    x, y = lp.labels[0], lp.labels[1]
    while True:
        passes += 1
        if C.lp_iterate(lp.seg, x, y) == 0 or passes > 10000:
            break
        x, y = y, x
    sp.record()
    sp.synchronize()
    t_lp = st.elapsed_time(sp) / 1e3
    out["label_propagation_rmat24_undirected"] = {
        "gteps_per_pass": g.E * passes / t_lp / 1e9, "ms_per_pass": t_lp / passes * 1e3,
        "passes": passes, "first_pass_bitexact_vs_oracle": bool(np.array_equal(first, want1)),
        "wall_s": time.time() - t0}
    del lp, graph, g
    torch.cuda.empty_cache()

    # 64-vector personalised PageRank (BF16 hi+lo) against 64 one-vector solves
    t0 = time.time()
    g = graphgen.rmat(22, 16, seed=1)
    graph = P.Graph(g.offsets, g.src, cluster_mode=0)
    nd = int((graph.outdeg > 0).sum().item())
    seeds = ppr_seeds(g)
    b = P.BatchedPPR(graph, bounds=_ppr_bounds(nd, graph.V, 1), planes=2)
    R, _ = b.run(seeds, ITERS)
    t_b = timed(lambda: (b.init(seeds), C.ppr_batched_iterate(b.ppr, graph.inv, DAMPING, ITERS,
                                                               b.rank)), reps=3)
    one = P.SegmentedPageRank(graph, bounds=P.plan_bounds(graph, 1, 32.0))
    one.run_ppr(int(seeds[0]), ITERS)
    t_1 = timed(lambda: [one.run_ppr(int(s_), ITERS) for s_ in seeds])
    want, bound = oracle.pagerank_bound(g.offsets, g.src, iters=ITERS, seed=int(seeds[0]),
                                        u_store=oracle.U_BF16X2)
    got = R[:, 0].cpu().numpy().astype(np.float64)
    err = np.abs(got - want)
    out["ppr64_rmat22"] = {
        "ms_per_64_vector_solve": t_b * 1e3, "ms_64_one_vector_solves": t_1 * 1e3,
        "speedup_vs_64_single": t_1 / t_b, "edge_vector_gteps": g.E * 64 * ITERS / t_b / 1e9,
        "column0_rel_l1": float(err.sum() / want.sum()),
        "column0_max_err_over_bound": float(np.max(err[bound > 0] / bound[bound > 0])),
        "column0_within_bound": bool(np.all(err <= bound)), "wall_s": time.time() - t0}
    del b, one, graph, g, R
    torch.cuda.empty_cache()

    # the 1,024-graph batch: one CUDA-graph-replayed launch against per-graph
    # launches, also replayed from a CUDA graph
    t0 = time.time()
    gs = graphgen.small_graph_batch(count=1024, seed=1, scale_lo=8, scale_hi=15)
    Etot = sum(len(x.src) for x in gs)
    bp = P.BatchedPageRank(gs)
    s2 = torch.cuda.Stream()
    s2.wait_stream(torch.cuda.current_stream())
    gb, gp = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    handles = [P.SegmentedPageRank(P.Graph(x.offsets, x.src, cluster_mode=None), 1) for x in gs]
    with torch.cuda.stream(s2):
        bp.run(ITERS)
        for h in handles[:4]:
            h.run(ITERS)
        torch.cuda.synchronize()
        with torch.cuda.graph(gb, stream=s2):
            C.pr_batch_run(bp.batch, ITERS, DAMPING, bp.rank)
        with torch.cuda.graph(gp, stream=s2, capture_error_mode="relaxed"):
            for h in handles:
                h.init()
                h.step(h.rank[0], h.contrib[0], h.rank[1], h.contrib[1], DAMPING, ITERS)
    torch.cuda.current_stream().wait_stream(s2)
    gb.replay()
    gp.replay()
    torch.cuda.synchronize()
    t_batch = timed(gb.replay, reps=5)
    t_per = timed(gp.replay, reps=3)
    rank = bp.rank.cpu().numpy()
    worst, inside = 0.0, True
    for i in range(0, 1024, 128):
        want, bound = oracle.pagerank_bound(gs[i].offsets, gs[i].src, iters=ITERS)
        e = np.abs(rank[bp.vbase[i]:bp.vbase[i + 1]].astype(np.float64) - want)
        worst = max(worst, float(np.max(e / bound)))
        inside &= bool(np.all(e <= bound))
    out["batched_1024_graphs"] = {
        "gteps": Etot * ITERS / t_batch / 1e9, "ms_per_solve": t_batch * 1e3,
        "per_graph_launches_cuda_graph_ms": t_per * 1e3, "speedup_vs_per_graph": t_per / t_batch,
        "sample_graphs": 8, "max_err_over_bound": worst, "within_bound": inside,
        "wall_s": time.time() - t0}
    del bp, handles, gb, gp, gs
    torch.cuda.empty_cache()

    # collaborative filtering: 10 sweeps at BF16 hi+lo; two FP32 sweeps vs FP64
    t0 = time.time()
    bpg = graphgen.bipartite(seed=1)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).cuda()  # noqa: E731
    uoff, uitem, urate = (dev(bpg.user_offsets, torch.int64), dev(bpg.items, torch.int32),
                          dev(bpg.ratings, torch.uint8))
    ioff = torch.empty(bpg.I + 1, dtype=torch.int64, device="cuda")
    iuser = torch.empty(bpg.R, dtype=torch.int32, device="cuda")
    irate = torch.empty(bpg.R, dtype=torch.uint8, device="cuda")
    C.cf_transpose(bpg.U, bpg.I, uoff, uitem, urate, ioff, iuser, irate)
    P0, Q0 = graphgen.cf_factors(bpg.U, bpg.I, 32, seed=1)
    P0, Q0 = P0.astype(np.float32), Q0.astype(np.float32)
    P0d, Q0d = dev(P0, torch.float32), dev(Q0, torch.float32)
    h = C.cf_create(bpg.U, bpg.I, 32, C.CF_BF16X2, uoff, uitem, urate, ioff, iuser, irate)
    C.cf_set_factors(h, P0d, Q0d)
    C.cf_sweep(h, 1, 0.05, 1e-3)
    C.cf_set_factors(h, P0d, Q0d)
    t_cf = timed(lambda: C.cf_sweep(h, 10, 0.05, 1e-3)) / 10
    del h
    # FP32: two sweeps, each checked entry by entry at 2,048 sampled users and
    # 64 sampled items against the oracle's rounding bound from the factors
    # the GPU held before it; then the drift from the oracle's trajectory
    h = C.cf_create(bpg.U, bpg.I, 32, C.CF_FP32, uoff, uitem, urate, ioff, iuser, irate)
    C.cf_set_factors(h, P0d, Q0d)
    Pg = torch.empty((bpg.U, 32), dtype=torch.float32, device="cuda")
    Qg = torch.empty((bpg.I, 32), dtype=torch.float32, device="cuda")
    io, iu, ir = oracle.item_major(bpg.U, bpg.I, bpg.user_offsets, bpg.items, bpg.ratings)
    rng = np.random.default_rng(3)
    ideg = np.diff(io)
    users = np.unique(rng.choice(bpg.U, 2048, replace=False))
    items = np.unique(rng.choice(np.flatnonzero(ideg <= 200_000), 64, replace=False))
    worst, outside = 0.0, 0
    Pw, Qw = P0.astype(np.float64), Q0.astype(np.float64)
    for _ in range(2):
        C.cf_get_factors(h, Pg, Qg)
        Pr, Qr = Pg.cpu().numpy().astype(np.float64), Qg.cpu().numpy().astype(np.float64)
        C.cf_sweep(h, 1, 0.05, 1e-3)
        C.cf_get_factors(h, Pg, Qg)
        Pn, Qn, _, bP, bQ, _ = oracle.cf_sweep_bound(bpg.U, bpg.I, bpg.user_offsets, bpg.items,
                                                     bpg.ratings, io, iu, ir, Pr, Qr, 0.05, 1e-3,
                                                     users=users, items=items)
        eP = np.abs(Pg.cpu().numpy()[users].astype(np.float64) - Pn[users]) / bP
        eQ = np.abs(Qg.cpu().numpy()[items].astype(np.float64) - Qn[items]) / bQ
        worst = max(worst, float(eP.max()), float(eQ.max()))
        outside += int(np.sum(eP > 1.0) + np.sum(eQ > 1.0))
        Pw, Qw, _ = oracle.cf_sweep(bpg.U, bpg.I, bpg.user_offsets, bpg.items, bpg.ratings, io,
                                    iu, ir, Pw, Qw, 0.05, 1e-3)
    rel = float(np.max(np.abs(Pg.cpu().numpy() - Pw)) / np.max(np.abs(Pw)))
    out["cf_netflix_shaped_k32"] = {
        "ms_per_sweep_bf16x2": t_cf * 1e3, "gteps_rating_sides": 2 * bpg.R / t_cf / 1e9,
        "fp32_sweeps_sampled_entries": 2 * 32 * (len(users) + len(items)),
        "fp32_sweeps_max_err_over_bound": worst, "fp32_sweeps_entries_outside_bound": outside,
        "fp32_two_sweeps_max_err_rel_to_max": rel, "fp32_drift_tolerance": 2e-6,
        "fp32_ok": bool(outside == 0 and rel <= 2e-6), "wall_s": time.time() - t0}
    del h, uoff, uitem, urate, ioff, iuser, irate, P0d, Q0d, Pg, Qg
    torch.cuda.empty_cache()

    # betweenness centrality from 12 sources on the headline graph; levels and
    # path counts must not depend on the direction (push only vs the switch)
    t0 = time.time()
    bc = P.Betweenness(graph25)
    S = ppr_seeds(g25, n=12)
    bc.run(S[:1])
    t_bc = timed(lambda: bc.run(S))
    bc.run(S[:1])
    l1, s1, _, inf1 = bc.source_state()
    C.bc_set_direction(bc.h, 0.0)
    bc.run(S[:1])
    l0, s0, _, inf0 = bc.source_state()
    out["betweenness_rmat25_12_sources"] = {
        "s_for_12_sources": t_bc, "gteps": 12 * g25.E / t_bc / 1e9,
        "levels": inf1["depth"], "push_levels": inf1["push_levels"],
        "pull_levels": inf1["pull_levels"],
        "levels_and_sigma_same_push_only": bool(torch.equal(l1, l0) and torch.equal(s1, s0)),
        "wall_s": time.time() - t0}
    del bc
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=25)
    ap.add_argument("--k", type=int, default=0, help="uniform segments (0: autotune)")
    ap.add_argument("--threads", type=int, default=1024, help="gather threads (with --k)")
    ap.add_argument("--ctas", type=int, default=1, help="gather blocks per SM (with --k)")
    ap.add_argument("--table", type=int, default=0,
                    help="shared table entries (with --k; with --plan, > 0 caps the table)")
    ap.add_argument("--plan", type=float, default=0.0,
                    help="use planned bounds with this min_avg_degree (skips the autotuner)")
    ap.add_argument("--merge-block", type=int, default=512)
    ap.add_argument("--overlap", type=int, default=0,
                    help="warps per block serving the L1/L2 segments inside the staged launch "
                         "(with --plan; the autotuner tries its own)")
    ap.add_argument("--affine", type=int, default=0,  # 1: head threshold = --plan
                    help="with --plan: the nested plan (cold range in table-sized segments "
                         "staged one block per segment)")
    ap.add_argument("--sweep", action="store_true", help="k = 1..64 sweep table")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the compact records of the other forms (LP, PPR, batch, CF, BC)")
    ap.add_argument("--workload", default="pagerank",
                    choices=["pagerank", "lp", "batched", "ppr", "cf", "bc", "qfactor",
                             "sweep", "profile"],
                    help="pagerank (the headline), lp (label propagation, RMAT-24 undirected) "
                         "or batched (1,024 small RMAT graphs, scales 8-15)")
    ap.add_argument("--graphs", type=int, default=1024, help="graphs of the batched workload")
    ap.add_argument("--dense", type=int, default=-1,
                    help="hub-block size for the tensor-core part of the ppr workload "
                         "(-1: autotune over 0, 4096 .. 32768; 0: none)")
    ap.add_argument("--arm", default="segmented",
                    choices=["segmented", "plain_random", "plain_clustered"],
                    help="the arm the profile workload runs")
    ap.add_argument("--iters", type=int, default=3, help="iterations of the profile workload")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "lp":
        return run_lp(args)
    if args.workload == "ppr":
        return run_ppr(args)
    if args.workload == "cf":
        return run_cf(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "bc":
        return run_bc(args)
    if args.workload == "qfactor":
        return run_qfactor(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "profile":
        return run_profile(args)

    import torch
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    import __graft_entry__
    __graft_entry__.build()
    from paper_1608_01362_gb300 import cagra as C
    from paper_1608_01362_gb300 import pipeline as P

    g, gen_s = make_graph(args.scale)
    V, E = g.V, g.E
    dev = torch.device("cuda", local)

    # ---- preprocessing (timed separately, as the paper does)
    torch.cuda.synchronize()
    t0 = time.time()
    graph = P.Graph(g.offsets, g.src, cluster_mode=0, device=dev)
    torch.cuda.synchronize()
    cluster_s = time.time() - t0

    if args.plan:
        best = {"kind": "plan", "threads": args.threads, "ctas": args.ctas,
                "min_avg_degree": args.plan, "table": args.table or -1, "overlap": args.overlap,
                "affine": args.affine}
        table = []
    elif args.k:
        best = {"kind": "uniform", "k": args.k, "threads": args.threads, "ctas": args.ctas,
                "table": args.table}
        table = []
    else:
        uk = (1, 2, 4, 8, 16, 32, 64) if args.sweep else (1, 4, 16)
        best, table = P.autotune_segments(graph, P.default_candidates(uniform_k=uk),
                                          merge_block=args.merge_block)
    torch.cuda.synchronize()
    t0 = time.time()
    pr = P.build_candidate(graph, best, merge_block=args.merge_block)
    torch.cuda.synchronize()
    seg_s = time.time() - t0
    info = pr.info
    best_k = info["num_segments"]

    stream = torch.cuda.current_stream()
    resid = torch.zeros(ITERS, dtype=torch.float64, device=dev)
    n_ev = args.steps * ITERS
    # events around the three launch groups of every timed iteration
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(n_ev)] for _ in range(4)]

    def one_step(events_at=None):
        """One PageRank solve (r_0 = 1/V, ITERS iterations) through the C ABI."""
        pr.init()
        rin, cin, rout, cout = pr.rank[0], pr.contrib[0], pr.rank[1], pr.contrib[1]
        for it in range(ITERS):
            e = None if events_at is None else events_at + it
            if e is not None:
                ev[0][e].record(stream)
            C.cg_seg_gather_phases(pr.seg, C.CG_OP_SUM_F32, cin, None, C.PHASE_STAGED)
            if e is not None:
                ev[1][e].record(stream)
            C.cg_seg_gather_phases(pr.seg, C.CG_OP_SUM_F32, cin, None,
                                   C.PHASE_CACHED | C.PHASE_FIXUP)
            if e is not None:
                ev[2][e].record(stream)
            C.pr_merge_update(pr.seg, graph.inv, rin, rout, cout, DAMPING, pr.dangling,
                              pr.dangling, resid[it:it + 1])
            if e is not None:
                ev[3][e].record(stream)
            rin, cin, rout, cout = rout, cout, rin, cin

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for s in range(args.steps):
        one_step(events_at=s * ITERS)
    stop.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if pg:
        pg.barrier()
    elapsed = start.elapsed_time(stop) / 1e3

    def mean_span(i, j):
        return float(np.mean([x.elapsed_time(y) for x, y in zip(ev[i], ev[j])])) / 1e3

    t_staged, t_cached, t_merge, t_iter_ev = (mean_span(0, 1), mean_span(1, 2), mean_span(2, 3),
                                              mean_span(0, 3))
    t_max = max_over_ranks(elapsed, pg)
    value = replica_value(E * ITERS * args.steps, world, t_max) / 1e9

    # ---- the timed configuration's own solve, for the parity check against the
    # FP64 oracle below
    rank_final, res = pr.run(ITERS)
    mass = float(rank_final.double().sum().item())
    rank_final_h = rank_final.cpu().numpy()

    # ---- e2e: public API with host buffers (pinned), copies inside the timed region
    rank_h = torch.full((V,), 1.0 / V, dtype=torch.float32).pin_memory()
    inv_dev = graph.inv
    out_h = torch.empty(V, dtype=torch.float32).pin_memory()
    rank_dev = torch.empty(V, dtype=torch.float32, device=dev)
    rank_cl = torch.empty_like(rank_dev)
    contrib_cl = torch.empty_like(rank_dev)
    e2e_steps = max(3, args.steps // 5)
    e_start = torch.cuda.Event(enable_timing=True)
    e_stop = torch.cuda.Event(enable_timing=True)

    def e2e_step():
        rank_dev.copy_(rank_h, non_blocking=True)                      # H2D: initial ranks
        C.cg_permute4(rank_dev, graph.old_of_new, rank_cl)             # original -> clustered
        C.pr_contrib(inv_dev, rank_cl, contrib_cl, pr.dangling)        # contrib, dangling mass
        C.pr_iterate(pr.seg, inv_dev, rank_cl, contrib_cl, pr.rank[1], pr.contrib[1], DAMPING,
                     ITERS, pr.dangling, resid)
        C.cg_permute4(pr.rank[1], graph.new_of_old, rank_dev)          # clustered -> original
        out_h.copy_(rank_dev, non_blocking=True)                       # D2H: result

    e2e_step()
    torch.cuda.synchronize()
    e_start.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e_stop.record(stream)
    torch.cuda.synchronize()
    e2e_t = max_over_ranks(e_start.elapsed_time(e_stop) / 1e3, pg)
    e2e_value = replica_value(E * ITERS * e2e_steps, world, e2e_t) / 1e9
    e2e_out = out_h.numpy().copy()

    # ---- comparisons on the same GPU: plain pull (original / clustered order), probe
    plain_orig_graph = P.Graph(g.offsets, g.src, cluster_mode=None, device=dev)
    plain_orig = P.PlainPageRank(plain_orig_graph)
    plain_orig.init()
    plain_orig.step(plain_orig.rank[0], plain_orig.contrib[0], plain_orig.rank[1],
                    plain_orig.contrib[1], DAMPING, 2)
    t_plain_orig = P.time_iterations(plain_orig, ITERS, reps=3)
    # the fourth variant of the paper's comparison: segmented in the original
    # (unclustered) order, the paper's uniform split at the best uniform k the
    # autotuner measured (4 when it did not run)
    uni = [r for r in table if r["candidate"]["kind"] == "uniform"]
    k_orig = int(min(uni, key=lambda r: r["s_per_iter"])["candidate"]["k"]) if uni else 4
    seg_orig = P.SegmentedPageRank(plain_orig_graph, k_orig)
    seg_orig.init()
    seg_orig.step(seg_orig.rank[0], seg_orig.contrib[0], seg_orig.rank[1], seg_orig.contrib[1],
                  DAMPING, 2)
    t_seg_orig = P.time_iterations(seg_orig, ITERS, reps=3)
    seg_orig.seg.close()
    del seg_orig
    plain_cl = P.PlainPageRank(graph)
    t_plain_cl = P.time_iterations(plain_cl, ITERS, reps=3)
    probe = P.PlainPageRank(graph, probe=True)
    t_probe = P.time_iterations(probe, ITERS, reps=3)
    seg_iter_s = t_max / (args.steps * ITERS)
    del plain_orig, plain_cl, probe, plain_orig_graph

    # ---- roofline: the unit is one PageRank iteration (every launch of the hot
    # path: staged gather, L1/L2 gather, fix-up, merge + vertex update) against
    # the method-independent byte count B_min = 4E + 28V (int64 offsets, int32
    # sources, FP32 vertex data), timed by events inside the timed region
    hbm, peak_kind = _peaks()
    rows = int(info["rows"])
    bmin = 4 * E + 28 * V
    achieved = bmin / t_iter_ev / 1e9
    traffic = _traffic_per_iteration(E, args.scale, best_k)
    # each launch against the ceiling of what it does: shared-memory lookups
    # (staged gather), random 4-byte L2 reads from the cold sources' table
    # (L1/L2 gather, fix-up included), HBM (merge + update: 8 B per subgraph
    # row, 20 B per vertex)
    staged_e = int(info["staged_edges"])
    cold_tab = 4 * max(2, min(1 << 24, V - int(info["staged_segments"]) * int(info["table_vertices"])))
    gp = gather_peaks(_probes(), [(4, cold_tab)], smem=True)
    m_bytes = 8 * rows + 20 * V
    per_launch = {
        "staged_gather": {"bound": "shared-memory random lookups", "unit": "G lookups/s",
                          "achieved": staged_e / t_staged / 1e9, "peak": gp["smem"],
                          "frac": staged_e / t_staged / 1e9 / gp["smem"]},
        "cached_gather_and_fixup": {
            "bound": "L2 random 4-byte reads", "unit": "GB/s", "table_bytes": cold_tab,
            "achieved": 4 * (E - staged_e) / t_cached / 1e9, "peak": gp[(4, cold_tab)],
            "frac": 4 * (E - staged_e) / t_cached / 1e9 / gp[(4, cold_tab)]},
        "merge_update": {"bound": "hbm", "unit": "GB/s", "algorithmic_bytes": m_bytes,
                         "achieved": m_bytes / t_merge / 1e9, "peak": hbm,
                         "frac": m_bytes / t_merge / 1e9 / hbm},
        "peaks_measured_by": "cg_measure_smem_lookups, cg_measure_row_gather in this run",
    }

    line = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"pagerank_rmat{args.scale}_directed_ef16_segmented_clustered",
                   "V": V, "E": E, "max_in_degree": int(np.diff(g.offsets).max()),
                   "max_out_degree": int(graph.outdeg.max().item()),
                   "iterations_per_step": ITERS, "damping": DAMPING,
                   "segments": best_k, "merge_block": args.merge_block, "q": info["q"],
                   "segmenting": best, "table_vertices": info["table_vertices"],
                   "staged_segments": info["staged_segments"],
                   "staged_edges": info["staged_edges"],
                   "ctas_per_sm": info["ctas_per_sm"],
                   "clustering": "descending out-degree (stable)",
                   "l2_policy": "inputs larger than L2 (2.1 GB edge stream per iteration)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "kernel": "one PageRank iteration (staged gather + L1/L2 gather + fix-up "
                               "+ merge/update launches)",
                     "algorithmic_bytes_per_launch": bmin, "peak_kind": peak_kind,
                     "avg_launch_ms": t_iter_ev * 1e3},
        "kernels_ms": {"staged_gather": t_staged * 1e3, "cached_gather_and_fixup": t_cached * 1e3,
                       "merge_update": t_merge * 1e3, "staged_edges": int(info["staged_edges"]),
                       "subgraph_rows": rows},
        "per_launch_bounds": per_launch,
        "gteps_at_hbm_peak": E / (bmin / (hbm * 1e9)) / 1e9,
        "comparisons": {
            "segmented_gteps": E / seg_iter_s / 1e9,
            "plain_original_order_gteps": E / t_plain_orig / 1e9,
            "segmented_original_order_gteps": E / t_seg_orig / 1e9,
            "segmented_original_order_k": k_orig,
            "plain_clustered_gteps": E / t_plain_cl / 1e9,
            "vertex0_probe_gteps": E / t_probe / 1e9,
            "speedup_vs_plain_original": t_plain_orig / seg_iter_s,
            "speedup_vs_plain_clustered": t_plain_cl / seg_iter_s,
        },
        "autotune": [{**r["candidate"], "k": r["k"], "q": round(r["q"], 4),
                      "gteps": round(E / r["s_per_iter"] / 1e9, 2)} for r in table],
        "preprocessing_s": {"generate_host": gen_s, "degrees_cluster_relabel": cluster_s,
                            "segment_build": seg_s},
        "rank_mass": mass,
        "e2e": {"value": e2e_value, "unit": "GTEPS", "h2d_bytes_per_step": 4 * V,
                "d2h_bytes_per_step": 4 * V, "steps": e2e_steps},
        "gpu_launches": args.steps * (2 + ITERS * (2 + int(info["staged_segments"] > 0) +
                                                   int(int(info["staged_edges"]) < E))),
        "clocks": clk,
    }
    if rank == 0 and not args.no_extras:
        line["sub_records"] = extras(g, graph)
    if rank == 0:
        # parity of exactly what was timed: the autotuned plan's 20-iteration
        # solve (and the end-to-end call's output) against the FP64 oracle,
        # vertex by vertex
        want, bound, secs, oracle_s = oracle_solution(g)
        line["parity"] = parity_report(rank_final_h, want, bound)
        line["parity"]["oracle_wall_s"] = oracle_s
        line["e2e"]["parity"] = parity_report(e2e_out, want, bound)
        line["e2e"]["result_ok"] = line["e2e"]["parity"]["ok"]
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_from(g, secs)
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
