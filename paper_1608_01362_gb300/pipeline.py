"""The call sequence a user makes, chained: out-degrees -> (optional)
frequency-based clustering -> CSR segmenting -> PageRank iterations, every
step a call into the CUDA library (no computation here).
"""
from __future__ import annotations

import numpy as np
import torch

from . import cagra as C


def _dev_csr(offsets, src, device):
    off = torch.as_tensor(offsets, dtype=torch.int64).to(device).contiguous()
    s = torch.as_tensor(src, dtype=torch.int32).to(device).contiguous()
    return off, s


class Graph:
    """An in-edge CSR on the GPU with its out-degrees, optionally renumbered
    hottest-first by frequency-based clustering (Section V)."""

    def __init__(self, offsets, src, cluster_mode: int | None = 0, device="cuda"):
        off, s = _dev_csr(offsets, src, device)
        self.device = torch.device(device)
        self.V = off.numel() - 1
        self.E = s.numel()
        outdeg = torch.empty(self.V, dtype=torch.int32, device=self.device)
        C.cg_out_degree(s, self.V, outdeg)
        self.cluster_mode = cluster_mode
        if cluster_mode is None:
            self.offsets, self.src, self.outdeg = off, s, outdeg
            self.new_of_old = self.old_of_new = None
        else:
            n2o = torch.empty(self.V, dtype=torch.int32, device=self.device)
            o2n = torch.empty_like(n2o)
            C.cg_cluster(outdeg, self.E, cluster_mode, n2o, o2n)
            noff = torch.empty_like(off)
            nsrc = torch.empty_like(s)
            C.cg_relabel_csr(off, s, n2o, o2n, noff, nsrc)
            nout = torch.empty_like(outdeg)
            C.cg_permute4(outdeg, o2n, nout)
            self.offsets, self.src, self.outdeg = noff, nsrc, nout
            self.new_of_old, self.old_of_new = n2o, o2n
        self.inv = torch.empty(self.V, dtype=torch.float32, device=self.device)
        C.cg_inv_outdeg(self.outdeg, self.inv)
        self._n2o_host = None

    def to_clustered_id(self, v: int) -> int:
        """Vertex ID in the numbering the kernels use."""
        if self.new_of_old is None:
            return int(v)
        if self._n2o_host is None:
            self._n2o_host = self.new_of_old.cpu().numpy()
        return int(self._n2o_host[int(v)])

    def rows_to_original(self, x):
        """[V, w] per-vertex rows in the clustered numbering -> original."""
        if self.new_of_old is None:
            return x
        out = torch.empty_like(x)
        C.cg_permute_rows(x, self.new_of_old, out)
        return out

    def to_original(self, x):
        """Vertex vector in the clustered numbering -> original numbering."""
        if self.new_of_old is None:
            return x
        out = torch.empty_like(x)
        C.cg_permute4(x, self.new_of_old, out)
        return out


class _PageRankBase:
    def __init__(self, graph: Graph):
        self.g = graph
        V, dev = graph.V, graph.device
        self.rank = [torch.empty(V, dtype=torch.float32, device=dev) for _ in range(2)]
        self.contrib = [torch.empty(V, dtype=torch.float32, device=dev) for _ in range(2)]
        self.dangling = torch.zeros(1, dtype=torch.float64, device=dev)

    def init(self):
        C.pr_init(self.g.inv, self.rank[0], self.contrib[0], self.dangling)

    def run(self, iterations: int = 20, damping: float = 0.85, resid=None):
        """r_0 = 1/V, then `iterations` iterations; returns (rank in original
        IDs, residual per iteration as a device FP64 tensor)."""
        if resid is None:
            resid = torch.zeros(iterations, dtype=torch.float64, device=self.g.device)
        self.init()
        self.step(self.rank[0], self.contrib[0], self.rank[1], self.contrib[1], damping,
                  iterations, resid)
        return self.g.to_original(self.rank[1]), resid


def plan_bounds(graph: Graph, ctas_per_sm: int = 1, min_avg_degree: float = 64.0,
                max_global_vertices: int = -1, table_vertices: int = -1):
    """Segment bounds for this GPU: shared-memory-sized segments over the hot
    (clustered) head, L2-sized segments over the cold rest (-1: half of the
    L2's bytes in 4-byte source values).  table_vertices
    (> 0) caps the shared table below its capacity, which leaves the rest of
    the SM's on-chip store to L1 (and to the misses L1 keeps in flight)."""
    H = C.pr_gather_table_capacity(ctas_per_sm)
    if table_vertices > 0:
        H = min(H, table_vertices)
    return C.pr_plan_bounds(graph.outdeg, H, min_avg_degree, max_global_vertices)


GATHER_SHAPES = ((1024, 1), (512, 2))  # staged gather (threads, blocks per SM)


class SegmentedPageRank(_PageRankBase):
    """PageRank through CSR segmenting (Algorithms 2-5)."""

    def __init__(self, graph: Graph, num_segments: int | None = None, merge_block: int = 512,
                 bounds=None, threads: int = 1024, ctas_per_sm: int = 1,
                 table_vertices: int = -1, overlap: int = 0, affine: float = 0.0):
        super().__init__(graph)
        if bounds is not None:
            bounds = np.asarray(bounds, dtype=np.int64)
            num_segments = len(bounds) - 1
        self.seg = C.pr_build_segments(graph.offsets, graph.src, num_segments, bounds=bounds,
                                       merge_block=merge_block)
        if (threads, ctas_per_sm, table_vertices) != (1024, 1, -1):
            C.pr_set_gather_config(self.seg, threads, ctas_per_sm, table_vertices)
        if overlap:
            C.pr_set_gather_overlap(self.seg, overlap)
        if affine:
            C.pr_set_gather_affine(self.seg, affine)

    @property
    def info(self):
        return self.seg.info

    def step(self, rank_in, contrib_in, rank_out, contrib_out, damping, iterations, resid=None):
        C.pr_iterate(self.seg, self.g.inv, rank_in, contrib_in, rank_out, contrib_out, damping,
                     iterations, self.dangling, resid)

    def run_ppr(self, seed: int, iterations: int = 20, damping: float = 0.85, resid=None):
        """Personalised PageRank of one seed (original ID): one-hot start,
        `iterations` iterations; returns (rank in original IDs, residuals)."""
        if resid is None:
            resid = torch.zeros(iterations, dtype=torch.float64, device=self.g.device)
        s = self.g.to_clustered_id(seed)
        C.pr_init_ppr(self.g.inv, s, self.rank[0], self.contrib[0], self.dangling)
        C.pr_iterate_ppr(self.seg, self.g.inv, self.rank[0], self.contrib[0], self.rank[1],
                         self.contrib[1], damping, iterations, s, self.dangling, resid)
        return self.g.to_original(self.rank[1]), resid


class BatchedPPR:
    """64 personalised PageRank vectors through one segmented graph.
    dense_hubs = h > 0 takes the block among vertices [0, h) (the hottest after
    clustering) out of the gather and onto the tensor cores."""

    def __init__(self, graph: Graph, num_segments: int | None = None, bounds=None,
                 planes: int = 2, merge_block: int = 512, dense_hubs: int = 0):
        self.g = graph
        if bounds is not None:
            bounds = np.asarray(bounds, dtype=np.int64)
            num_segments = len(bounds) - 1
        off, src = graph.offsets, graph.src
        self.dense_hubs = int(dense_hubs)
        if self.dense_hubs:
            h = self.dense_hubs
            self.rest_off = torch.empty_like(off)
            rest = torch.empty_like(src)
            self.bits = torch.empty(h * (h // 32), dtype=torch.int32, device=graph.device)
            er = C.cg_split_hub_block(off, src, h, self.rest_off, rest, self.bits)
            self.rest_src = rest[:er].contiguous()
            off, src = self.rest_off, self.rest_src
        self.seg = C.pr_build_segments(off, src, num_segments, bounds=bounds,
                                       merge_block=merge_block)
        self.ppr = C.ppr_batched_create(self.seg, planes)
        if self.dense_hubs:
            C.ppr_batched_attach_dense(self.ppr, self.dense_hubs, self.bits)
        self.rank = torch.empty((graph.V, C.PPR_COLUMNS), dtype=torch.float32,
                                device=graph.device)
        self.resid = torch.zeros(C.PPR_COLUMNS, dtype=torch.float64, device=graph.device)

    def init(self, seeds):
        """seeds: 64 vertex IDs (original numbering)."""
        C.ppr_batched_init(self.ppr, self.g.inv,
                           [self.g.to_clustered_id(int(s)) for s in seeds])

    def run(self, seeds, iterations: int = 20, damping: float = 0.85):
        """Returns (R [V, 64] in original vertex IDs, per-column residual of the
        last iteration as a device FP64 tensor)."""
        self.init(seeds)
        C.ppr_batched_iterate(self.ppr, self.g.inv, damping, iterations, self.rank,
                              self.resid if iterations >= 2 else None)
        return self.g.rows_to_original(self.rank), self.resid


class PlainPageRank(_PageRankBase):
    """The plain pull baseline (Algorithm 1) over the whole CSR."""

    def __init__(self, graph: Graph, probe: bool = False):
        super().__init__(graph)
        self.plain = C.pr_plain_create(graph.offsets, graph.src)
        self.probe = probe

    def step(self, rank_in, contrib_in, rank_out, contrib_out, damping, iterations, resid=None):
        C.pr_iterate_plain(self.plain, self.g.inv, rank_in, contrib_in, rank_out, contrib_out,
                           damping, iterations, self.dangling, resid, probe=self.probe)


def time_iterations(pr, iterations: int = 3, damping: float = 0.85, reps: int = 1) -> float:
    """Median seconds per PageRank iteration of `pr` (CUDA events)."""
    times = []
    for _ in range(reps):
        pr.init()
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record()
        pr.step(pr.rank[0], pr.contrib[0], pr.rank[1], pr.contrib[1], damping, iterations)
        stop.record()
        stop.synchronize()
        times.append(start.elapsed_time(stop) / 1e3 / iterations)
    times.sort()
    return times[len(times) // 2]


def default_candidates(uniform_k=(1, 4), shapes=GATHER_SHAPES,
                       min_deg=(4.0, 16.0, 24.0, 32.0, 48.0, 64.0, 256.0),
                       tables=(-1, 0), affine_deg=(16.0, 24.0, 32.0, 48.0)):
    """Autotuner search space: the paper's uniform split into k segments, and
    the GPU plan (shared-memory segments over the hot head, L2 segments over
    the rest), at several gather launch shapes, shared-table sizes and
    staging thresholds; and the nested plan (the cold rest cut into
    table-sized segments staged one block per segment) at the head
    thresholds affine_deg.  A smaller table leaves more of the SM's on-chip
    memory to the L1 cache, which serves the reads the table does not."""
    out = [{"kind": "uniform", "k": k, "threads": 1024, "ctas": 1, "table": tb}
           for k in uniform_k for tb in tables]
    out += [{"kind": "plan", "threads": t, "ctas": c, "min_avg_degree": m, "table": -1}
            for (t, c) in shapes for m in min_deg]
    out += [{"kind": "plan", "threads": 1024, "ctas": 1, "min_avg_degree": m, "table": -1,
             "affine": 1} for m in affine_deg]
    return out


def _build(graph, cand, merge_block):
    t, c, tb = cand.get("threads", 1024), cand.get("ctas", 1), cand.get("table", -1)
    if cand["kind"] == "uniform":
        return SegmentedPageRank(graph, cand["k"], merge_block=merge_block, threads=t,
                                 ctas_per_sm=c, table_vertices=tb)
    # the nested plan cuts the cold range into table-sized segments, staged one
    # block per segment after the head (head threshold = min_avg_degree)
    affine = cand["min_avg_degree"] if cand.get("affine", 0) else 0.0
    mg = C.pr_gather_table_capacity(c) if affine else -1
    b = plan_bounds(graph, c, cand["min_avg_degree"], max_global_vertices=mg, table_vertices=tb)
    return SegmentedPageRank(graph, bounds=b, merge_block=merge_block, threads=t, ctas_per_sm=c,
                             table_vertices=tb, overlap=cand.get("overlap", 0), affine=affine)


def autotune_segments(graph: Graph, candidates=None, merge_block: int = 512,
                      iterations: int = 3, reps: int = 3):
    """Pick the segmenting by measuring a few iterations of each candidate
    (Section III-D's trade-off: smaller segments confine the random reads to
    a smaller, faster memory but raise the expansion factor q and the merge
    traffic).  Returns (best candidate, list of {candidate, s_per_iter, q, k})."""
    if candidates is None:
        candidates = default_candidates()
    results = []
    best = None
    for cand in candidates:
        if cand["kind"] == "uniform" and cand["k"] > graph.V:
            continue
        pr = _build(graph, cand, merge_block)
        pr.init()
        pr.step(pr.rank[0], pr.contrib[0], pr.rank[1], pr.contrib[1], 0.85, 1)  # warm-up
        t = time_iterations(pr, iterations, reps=reps)
        inf = pr.info
        results.append({"candidate": cand, "s_per_iter": t, "q": inf["q"],
                        "k": inf["num_segments"], "table_vertices": inf["table_vertices"]})
        if best is None or t < best[1]:
            best = (cand, t)
        pr.seg.close()
        del pr
    return best[0], results


def build_candidate(graph: Graph, cand: dict, merge_block: int = 512) -> SegmentedPageRank:
    return _build(graph, cand, merge_block)


class LabelPropagation:
    """Min-label propagation (connected components of a symmetric graph)
    through the segmented structure.  Labels start at each vertex's original
    ID, carried through the clustering permutation, so the result is the
    smallest original ID in each component whatever the renumbering."""

    def __init__(self, graph: Graph, num_segments: int | None = None, bounds=None,
                 merge_block: int = 512, threads: int = 1024, ctas_per_sm: int = 1,
                 table_vertices: int = -1, overlap: int = 0, affine: float = 0.0):
        self.g = graph
        if bounds is not None:
            bounds = np.asarray(bounds, dtype=np.int64)
            num_segments = len(bounds) - 1
        self.seg = C.pr_build_segments(graph.offsets, graph.src, num_segments, bounds=bounds,
                                       merge_block=merge_block)
        if (threads, ctas_per_sm, table_vertices) != (1024, 1, -1):
            C.pr_set_gather_config(self.seg, threads, ctas_per_sm, table_vertices)
        if overlap:
            C.pr_set_gather_overlap(self.seg, overlap)
        if affine:
            C.pr_set_gather_affine(self.seg, affine)
        V = graph.V
        self.labels = [torch.empty(V, dtype=torch.int32, device=graph.device) for _ in range(2)]

    def init(self):
        if self.g.old_of_new is None:
            self.labels[0].copy_(torch.arange(self.g.V, dtype=torch.int32,
                                              device=self.g.device))
        else:
            self.labels[0].copy_(self.g.old_of_new)
        return self.labels[0]

    def run(self, max_passes: int = 1 << 20):
        """Returns (labels in original IDs, passes, changes per pass)."""
        lab = self.init()
        passes, changes = C.lp_run(self.seg, lab, max_passes)
        return self.g.to_original(lab), passes, changes


class Betweenness:
    """Betweenness centrality from a set of sources (Brandes over frontiers)
    on a Graph (clustered or not): the out-edge CSR is built on the GPU by
    cg_transpose_csr.  Sources and results are in original vertex IDs."""

    def __init__(self, graph: Graph, alpha: float | None = None):
        self.g = graph
        self.out_off = torch.empty_like(graph.offsets)
        self.out_dst = torch.empty_like(graph.src)
        C.cg_transpose_csr(graph.offsets, graph.src, self.out_off, self.out_dst)
        self.h = C.bc_create(graph.offsets, graph.src, self.out_off, self.out_dst)
        if alpha is not None:
            C.bc_set_direction(self.h, alpha)
        self.bc = torch.zeros(graph.V, dtype=torch.float64, device=graph.device)

    def run(self, sources):
        """Centrality of every vertex from `sources` (original IDs), FP64,
        in original vertex IDs."""
        self.bc.zero_()
        C.bc_run(self.h, [self.g.to_clustered_id(int(s)) for s in sources], self.bc)
        return self.to_original8(self.bc)

    def to_original8(self, x):
        if self.g.new_of_old is None:
            return x
        out = torch.empty_like(x)
        C.cg_permute8(x, self.g.new_of_old, out)
        return out

    def source_state(self):
        """(level int32, sigma, delta) of the last source, original IDs."""
        V, dev = self.g.V, self.g.device
        lev = torch.empty(V, dtype=torch.int32, device=dev)
        sig = torch.empty(V, dtype=torch.float64, device=dev)
        dl = torch.empty(V, dtype=torch.float64, device=dev)
        info = C.bc_source_state(self.h, lev, sig, dl)
        return self.g.to_original(lev), self.to_original8(sig), self.to_original8(dl), info


def concat_graphs(graphs):
    """Concatenate in-edge CSRs (numpy offsets int64, src int32, local IDs)
    into the batched layout: (vbase, global offsets, local sources)."""
    vbase = np.zeros(len(graphs) + 1, dtype=np.int64)
    ebase = np.zeros(len(graphs) + 1, dtype=np.int64)
    for i, g in enumerate(graphs):
        vbase[i + 1] = vbase[i] + (len(g.offsets) - 1)
        ebase[i + 1] = ebase[i] + len(g.src)
    offsets = np.empty(vbase[-1] + 1, dtype=np.int64)
    src = np.empty(ebase[-1], dtype=np.int32)
    for i, g in enumerate(graphs):
        offsets[vbase[i]:vbase[i + 1]] = np.asarray(g.offsets[:-1]) + ebase[i]
        src[ebase[i]:ebase[i + 1]] = g.src
    offsets[-1] = ebase[-1]
    return vbase, offsets, src


class BatchedPageRank:
    """PageRank of many small graphs in one persistent launch."""

    def __init__(self, graphs, device="cuda", threads: int = 1024):
        vbase, offsets, src = concat_graphs(graphs)
        self.device = torch.device(device)
        self.vbase = vbase
        self.offsets = torch.as_tensor(offsets).to(self.device)
        self.src = torch.as_tensor(src).to(self.device)
        self.batch = C.pr_batch_create(vbase, self.offsets, self.src)
        if threads != 1024:
            C.pr_batch_set_threads(self.batch, threads)
        self.rank = torch.empty(int(vbase[-1]), dtype=torch.float32, device=self.device)

    def run(self, iterations: int = 20, damping: float = 0.85, resid=None):
        C.pr_batch_run(self.batch, iterations, damping, self.rank, resid)
        return self.rank
