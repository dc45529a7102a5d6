"""Parity of the CUDA path (through the C ABI) against the FP64 oracle:
degrees, clustering, renumbering and segment construction bit for bit;
PageRank within 1e-5 relative L1 after 20 iterations (FP32 vs FP64)."""
import numpy as np
import pytest

import graphgen
import oracle as O
from parity import assert_gather_merge_exact, check_pagerank, pagerank_ref

pytestmark = pytest.mark.gpu

# FP32 residual sum |r' - r|: each term carries rounding of order 2^-24 (|r'| + |r|), so
# the residual cannot resolve below about 2 * 2^-24 * (sum r' + sum r) = 2.4e-7.
RESID_FLOOR = 2.4e-7


def resid_ok(got, want):
    return bool(np.all(np.abs(got - want) <= 1e-2 * want + RESID_FLOOR))


@pytest.fixture(scope="module")
def C():
    import torch
    assert torch.cuda.is_available()
    from paper_1608_01362_gb300 import build, cagra
    build.build()
    cagra.load()
    return cagra


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def _dev(torch, a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()



@pytest.fixture(scope="module")
def rmat16():
    return graphgen.rmat(16, 16, seed=1)


def _special_graphs():
    out = {}
    out["single"] = graphgen.from_edges(1, [], [])
    out["two_isolated"] = graphgen.from_edges(2, [], [])
    n = 5000  # in-star: one row much longer than a tile (carry fix-up across tiles)
    out["in_star"] = graphgen.from_edges(n + 1, np.arange(1, n + 1), np.zeros(n, dtype=int))
    out["out_star"] = graphgen.from_edges(n + 1, np.zeros(n, dtype=int), np.arange(1, n + 1))
    m = 3000
    out["cycle"] = graphgen.from_edges(m, np.arange(m), (np.arange(m) + 1) % m)
    rng = np.random.default_rng(5)
    out["ragged"] = graphgen.from_edges(777, rng.integers(0, 777, 5000) ** 1,
                                        (rng.integers(0, 777, 5000) ** 2) % 777)
    return out


# ------------------------------------------------------------------ integer work (bit-exact)

def test_out_degree_bitexact(C, torch_mod, rmat16):
    torch = torch_mod
    g = rmat16
    od = torch.empty(g.V, dtype=torch.int32, device="cuda")
    C.cg_out_degree(_dev(torch, g.src, torch.int32), g.V, od)
    assert np.array_equal(od.cpu().numpy(), O.out_degree(g.offsets, g.src))


@pytest.mark.parametrize("mode", [0, 1])
def test_cluster_and_relabel_bitexact(C, torch_mod, rmat16, mode):
    torch = torch_mod
    g = rmat16
    od_ref = O.out_degree(g.offsets, g.src)
    n2o_ref, o2n_ref = O.cluster(od_ref, mode, E=g.E)
    od = _dev(torch, od_ref, torch.int32)
    n2o = torch.empty(g.V, dtype=torch.int32, device="cuda")
    o2n = torch.empty_like(n2o)
    C.cg_cluster(od, g.E, mode, n2o, o2n)
    assert np.array_equal(o2n.cpu().numpy(), o2n_ref)
    assert np.array_equal(n2o.cpu().numpy(), n2o_ref)
    off, src = _dev(torch, g.offsets, torch.int64), _dev(torch, g.src, torch.int32)
    noff, nsrc = torch.empty_like(off), torch.empty_like(src)
    C.cg_relabel_csr(off, src, n2o, o2n, noff, nsrc)
    roff, rsrc = O.relabel(g.offsets, g.src, n2o_ref, o2n_ref)
    assert np.array_equal(noff.cpu().numpy(), roff) and np.array_equal(nsrc.cpu().numpy(), rsrc)


def test_cluster_large_keys_and_ties(C, torch_mod):
    torch = torch_mod
    rng = np.random.default_rng(3)
    V = 300_000
    od = np.where(rng.random(V) < 0.01, rng.integers(0, 2_000_000, V), rng.integers(0, 4, V))
    od = od.astype(np.int32)
    _, o2n_ref = O.cluster(od, 0)
    n2o = torch.empty(V, dtype=torch.int32, device="cuda")
    o2n = torch.empty_like(n2o)
    C.cg_cluster(_dev(torch, od, torch.int32), int(od.sum()), 0, n2o, o2n)
    assert np.array_equal(o2n.cpu().numpy(), o2n_ref)


def _check_segments(C, torch, offsets, src, k, B, bounds=None):
    ref = O.build_segments(offsets, src, k=k, B=B, bounds=bounds)
    seg = C.pr_build_segments(_dev(torch, offsets, torch.int64), _dev(torch, src, torch.int32), k,
                              bounds=bounds, merge_block=B)
    got = C.cg_segmented_export(seg)
    for name in ("bounds", "row_base", "edge_base", "row_ptr", "col", "idx_map", "block_start"):
        want = getattr(ref, name)
        assert np.array_equal(got[name], want), f"{name} differs (k={k}, B={B})"
    info = seg.info
    assert info["rows"] == ref.rows and abs(info["q"] - ref.q) < 1e-12
    return seg


@pytest.mark.parametrize("k,B", [(1, 4096), (2, 1024), (4, 4096), (7, 333), (16, 4096),
                                 (64, 6144), (1024, 64)])
def test_segments_bitexact_rmat16(C, torch_mod, rmat16, k, B):
    _check_segments(C, torch_mod, rmat16.offsets, rmat16.src, k, B)


def test_segments_bitexact_clustered_and_nonuniform(C, torch_mod, rmat16):
    g = rmat16
    n2o, o2n = O.cluster(O.out_degree(g.offsets, g.src), 0)
    off, src = O.relabel(g.offsets, g.src, n2o, o2n)
    _check_segments(C, torch_mod, off, src, 8, 2048)
    bounds = np.array([0, 1000, 1000, 20000, 20001, g.V], dtype=np.int64)  # empty + 1-vertex
    _check_segments(C, torch_mod, off, src, 5, 4096, bounds=bounds)


@pytest.mark.parametrize("name", list(_special_graphs().keys()))
def test_segments_bitexact_special(C, torch_mod, name):
    g = _special_graphs()[name]
    for k in (1, 3):
        if k <= g.V:
            _check_segments(C, torch_mod, g.offsets, g.src, k, 7)


def test_build_rejects_bad_input(C, torch_mod):
    torch = torch_mod
    off = _dev(torch, np.array([0, 2, 1, 3]), torch.int64)   # not monotone
    src = _dev(torch, np.array([0, 1, 2]), torch.int32)
    with pytest.raises(C.CagraError, match="INVALID_ARG"):
        C.pr_build_segments(off, src, 1)
    off = _dev(torch, np.array([0, 1, 2, 3]), torch.int64)
    src = _dev(torch, np.array([0, 7, 2]), torch.int32)      # source out of range
    with pytest.raises(C.CagraError, match="INVALID_ARG"):
        C.pr_build_segments(off, src, 1)
    src = _dev(torch, np.array([0, 1, 2]), torch.int32)
    with pytest.raises(C.CagraError, match="num_segments"):
        C.pr_build_segments(off, src, 0)
    with pytest.raises(C.CagraError, match="bounds"):
        C.pr_build_segments(off, src, 2, bounds=np.array([0, 2, 1]))


# ------------------------------------------------------------------ gather / merge alone

@pytest.mark.parametrize("k", [1, 5])
def test_seg_gather_and_merge(C, torch_mod, rmat16, k):
    torch = torch_mod
    g = rmat16
    ref = O.build_segments(g.offsets, g.src, k=k, B=1000)
    seg = C.pr_build_segments(_dev(torch, g.offsets, torch.int64), _dev(torch, g.src, torch.int32),
                              k, merge_block=1000)
    rng = np.random.default_rng(k)
    x = rng.random(g.V).astype(np.float32)
    interm = torch.empty(ref.rows, dtype=torch.float32, device="cuda")
    C.cg_seg_gather(seg, C.CG_OP_SUM_F32, _dev(torch, x, torch.float32), interm)
    want = np.array([x[ref.col[ref.row_ptr[i]:ref.row_ptr[i + 1]]].astype(np.float64).sum()
                     for i in range(ref.rows)])
    got = interm.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - want) / np.maximum(want, 1e-30)) < 1e-5
    out = torch.empty(g.V, dtype=torch.float32, device="cuda")
    C.merge(seg, C.CG_OP_SUM_F32, interm, out)
    dense = np.zeros(g.V)
    np.add.at(dense, ref.idx_map, got)
    assert np.max(np.abs(out.cpu().numpy() - dense) / np.maximum(dense, 1e-30)) < 1e-6
    # integer min: bit-exact
    lab = rng.permutation(g.V).astype(np.int32)
    imin = torch.empty(ref.rows, dtype=torch.int32, device="cuda")
    C.cg_seg_gather(seg, C.CG_OP_MIN_I32, _dev(torch, lab, torch.int32), imin)
    want = np.array([lab[ref.col[ref.row_ptr[i]:ref.row_ptr[i + 1]]].min()
                     for i in range(ref.rows)])
    assert np.array_equal(imin.cpu().numpy(), want)
    omin = torch.empty(g.V, dtype=torch.int32, device="cuda")
    C.merge(seg, C.CG_OP_MIN_I32, imin, omin)
    dm = np.full(g.V, 2**31 - 1, dtype=np.int64)
    np.minimum.at(dm, ref.idx_map, want)
    assert np.array_equal(omin.cpu().numpy(), dm)


# ------------------------------------------------------------------ PageRank

def _pagerank_gpu(torch, g, k=None, cluster=0, iters=20, B=4096, bounds=None, probe=False):
    from paper_1608_01362_gb300 import pipeline as P
    graph = P.Graph(g.offsets, g.src, cluster_mode=cluster)
    pr = P.PlainPageRank(graph, probe=probe) if k is None else \
        P.SegmentedPageRank(graph, k, merge_block=B, bounds=bounds)
    rank, resid = pr.run(iterations=iters)
    torch.cuda.synchronize()
    return rank.cpu().numpy(), resid.cpu().numpy(), pr


@pytest.fixture(scope="module")
def rmat16_oracle(rmat16):
    """(rank, residuals, per-vertex FP32 rounding bound) after 20 iterations."""
    want, want_resid = O.pagerank(rmat16.offsets, rmat16.src, iters=20)
    r, bound = pagerank_ref(rmat16)
    assert np.array_equal(r, want)
    return want, want_resid, bound


@pytest.mark.parametrize("cluster", [None, 0])
def test_plain_pagerank_parity(C, torch_mod, rmat16, rmat16_oracle, cluster):
    rank, resid, _ = _pagerank_gpu(torch_mod, rmat16, None, cluster)
    want, want_resid, bound = rmat16_oracle
    check_pagerank(rank, want, bound, what=f"plain cluster={cluster}")
    assert abs(rank.astype(np.float64).sum() - 1.0) < 1e-4
    assert resid_ok(resid, want_resid)


@pytest.mark.parametrize("k,cluster,B", [(1, None, 4096), (2, None, 4096), (4, 0, 4096),
                                         (8, 0, 1024), (16, 1, 4096), (64, 0, 6144),
                                         (1024, 0, 256)])
def test_segmented_pagerank_parity(C, torch_mod, rmat16, rmat16_oracle, k, cluster, B):
    rank, resid, pr = _pagerank_gpu(torch_mod, rmat16, k, cluster, B=B)
    want, want_resid, bound = rmat16_oracle
    check_pagerank(rank, want, bound, what=f"segmented k={k} cluster={cluster} B={B}")
    assert resid_ok(resid, want_resid)
    assert pr.info["num_segments"] == k
    rows, q, nbytes = pr.seg.stats()
    assert (rows, q, nbytes) == (pr.info["rows"], pr.info["q"], pr.info["device_bytes"])
    assert q <= min(k, rmat16.E / rmat16.V)


@pytest.mark.parametrize("k,cluster,B", [(1, None, 4096), (3, 0, 1000), (16, 1, 512),
                                         (64, 0, 6144), (1024, 0, 256)])
def test_gather_merge_exact_on_integers(C, torch_mod, rmat16, k, cluster, B):
    """Gather + merge of small integers equals the exact in-neighbour sums
    bit for bit (one dropped or duplicated edge anywhere would show)."""
    from paper_1608_01362_gb300 import pipeline as P
    graph = P.Graph(rmat16.offsets, rmat16.src, cluster_mode=cluster)
    pr = P.SegmentedPageRank(graph, k, merge_block=B)
    assert_gather_merge_exact(torch_mod, C, rmat16, graph, pr.seg, f"k={k} cluster={cluster}")


@pytest.mark.parametrize("name", ["in_star", "out_star", "cycle", "ragged"])
def test_gather_merge_exact_special_graphs(C, torch_mod, name):
    from paper_1608_01362_gb300 import pipeline as P
    g = _special_graphs()[name]
    graph = P.Graph(g.offsets, g.src, cluster_mode=0)
    for k in (1, 3):
        pr = P.SegmentedPageRank(graph, k, merge_block=64)
        assert_gather_merge_exact(torch_mod, C, g, graph, pr.seg, f"{name} k={k}")


def test_gather_merge_exact_every_autotuner_candidate(C, torch_mod, rmat16):
    """Every plan the autotuner may pick (planned bounds at each staging
    threshold and launch shape, the uniform splits, both table settings)."""
    from paper_1608_01362_gb300 import pipeline as P
    graph = P.Graph(rmat16.offsets, rmat16.src, cluster_mode=0)
    for cand in P.default_candidates(uniform_k=(1, 2, 4, 8, 16, 32, 64)):
        pr = P.build_candidate(graph, cand)
        assert_gather_merge_exact(torch_mod, C, rmat16, graph, pr.seg, str(cand))
        pr.seg.close()


def test_segmented_nonuniform_bounds(C, torch_mod, rmat16, rmat16_oracle):
    V = rmat16.V
    bounds = np.array([0, 4096, 4096, 30000, V], dtype=np.int64)
    rank, _, _ = _pagerank_gpu(torch_mod, rmat16, 4, 0, bounds=bounds)
    check_pagerank(rank, rmat16_oracle[0], rmat16_oracle[2], what="non-uniform bounds")


@pytest.mark.parametrize("name", list(_special_graphs().keys()))
def test_pagerank_special_graphs(C, torch_mod, name):
    g = _special_graphs()[name]
    want, bound = pagerank_ref(g)
    for k in (None, 1, 3):
        if k is not None and k > g.V:
            continue
        rank, _, _ = _pagerank_gpu(torch_mod, g, k, 0, B=64)
        check_pagerank(rank, want, bound, what=f"{name} k={k}")


def test_single_iteration_and_ping_pong(C, torch_mod, rmat16):
    """iterations = 1, 2, 3 land in the output buffers and match the oracle."""
    for it in (1, 2, 3):
        want, bound = pagerank_ref(rmat16, iters=it)
        rank, resid, _ = _pagerank_gpu(torch_mod, rmat16, 4, 0, iters=it)
        check_pagerank(rank, want, bound, what=f"iterations={it}")
        assert resid.shape == (it,)


def test_probe_reads_vertex_zero_only(C, torch_mod):
    """The lower-bound probe gathers contrib[0] for every edge (Fig. 1)."""
    torch = torch_mod
    g = graphgen.rmat(12, 8, seed=2)
    from paper_1608_01362_gb300 import pipeline as P
    graph = P.Graph(g.offsets, g.src, cluster_mode=None)
    pr = P.PlainPageRank(graph, probe=True)
    pr.init()
    pr.step(pr.rank[0], pr.contrib[0], pr.rank[1], pr.contrib[1], 0.85, 1)
    got = pr.rank[1].cpu().numpy().astype(np.float64)
    od = O.out_degree(g.offsets, g.src)
    c0 = (1.0 / g.V) / od[0] if od[0] else 0.0
    D = (od == 0).sum() / g.V
    want = 0.15 / g.V + 0.85 * (np.diff(g.offsets) * c0 + D / g.V)
    assert np.max(np.abs(got - want) / want) < 1e-5


def test_pagerank_rejects_aliasing(C, torch_mod, rmat16):
    torch = torch_mod
    from paper_1608_01362_gb300 import pipeline as P
    graph = P.Graph(rmat16.offsets, rmat16.src, cluster_mode=None)
    pr = P.SegmentedPageRank(graph, 2)
    pr.init()
    with pytest.raises(C.CagraError, match="alias"):
        pr.step(pr.rank[0], pr.contrib[0], pr.rank[0], pr.contrib[1], 0.85, 1)
    with pytest.raises(C.CagraError, match="iterations"):
        pr.step(pr.rank[0], pr.contrib[0], pr.rank[1], pr.contrib[1], 0.85, 0)


def test_deterministic_repeat(C, torch_mod, rmat16):
    a, ra, _ = _pagerank_gpu(torch_mod, rmat16, 4, 0)
    b, rb, _ = _pagerank_gpu(torch_mod, rmat16, 4, 0)
    assert np.array_equal(a, b) and np.array_equal(ra, rb)


# ------------------------------------------------------------------ shared-table / planned segments

@pytest.mark.parametrize("threads,ctas,table", [(1024, 1, 0), (1024, 1, 100), (1024, 1, -1),
                                               (512, 2, -1), (512, 1, 5000), (512, 2, 300)])
def test_gather_table_configs(C, torch_mod, rmat16, rmat16_oracle, threads, ctas, table):
    """The shared-memory table (whole segment or its hot head) and the launch
    shape change where values are read from, not the result."""
    from paper_1608_01362_gb300 import pipeline as P
    graph = P.Graph(rmat16.offsets, rmat16.src, cluster_mode=0)
    for k in (1, 3, 40):
        pr = P.SegmentedPageRank(graph, k, threads=threads, ctas_per_sm=ctas,
                                 table_vertices=table)
        info = pr.info
        assert info["ctas_per_sm"] == ctas and info["gather_threads"] == threads
        if table >= 0:
            assert info["table_vertices"] <= table
        if info["staged_segments"] == 0:
            assert info["table_vertices"] == 0
        rank, resid = pr.run(20)
        check_pagerank(rank.cpu().numpy(), rmat16_oracle[0], rmat16_oracle[2],
                       what=f"threads={threads} ctas={ctas} table={table} k={k}")


def test_gather_config_rejects_bad_shape(C, torch_mod, rmat16):
    from paper_1608_01362_gb300 import pipeline as P
    graph = P.Graph(rmat16.offsets, rmat16.src, cluster_mode=0)
    pr = P.SegmentedPageRank(graph, 2)
    assert pr.info["gather_threads"] == 1024 and pr.info["ctas_per_sm"] == 1
    with pytest.raises(C.CagraError, match="threads"):
        C.pr_set_gather_config(pr.seg, 256, 1, -1)
    with pytest.raises(C.CagraError, match="ctas_per_sm"):
        C.pr_set_gather_config(pr.seg, 1024, 2, -1)


def _overlap_graphs():
    gs = {"rmat16": graphgen.rmat(16, 16, seed=1)}
    gs.update({n: g for n, g in _special_graphs().items() if n in ("in_star", "out_star", "ragged")})
    # 600 sources of out-degree 8 (a staged head) and 3000 of out-degree 1 that
    # all point at vertex 0: a row of 3000 edges inside the L1/L2 segments, so
    # it spans many queue chunks and is completed through their carries
    rng = np.random.default_rng(9)
    hot = np.repeat(np.arange(600), 8)
    src = np.concatenate([hot, np.arange(600, 3600)])
    dst = np.concatenate([rng.integers(1, 3600, hot.size), np.zeros(3000, dtype=np.int64)])
    gs["cold_hub"] = graphgen.from_edges(3600, src, dst)
    return gs


@pytest.mark.parametrize("name", ["rmat16", "in_star", "out_star", "ragged", "cold_hub"])
def test_gather_overlap_bit_identical(C, torch_mod, name):
    """One launch serving staged and L1/L2 segments side by side (warps split
    per block, a chunk queue for the L1/L2 side) gives the same row sums, bit
    for bit, as the two launches, for every split; PageRank and min-label
    gathers through it too."""
    torch = torch_mod
    from paper_1608_01362_gb300 import pipeline as P
    g = _overlap_graphs()[name]
    graph = P.Graph(g.offsets, g.src, cluster_mode=0)
    # a staged head of 512-vertex segments and a cold rest of small L1/L2 segments
    b = C.pr_plan_bounds(graph.outdeg, 512, 2.0, 3000)
    seg = C.pr_build_segments(graph.offsets, graph.src, len(b) - 1, bounds=b)
    info = seg.info
    rows = info["rows"]
    rng = np.random.default_rng(3)
    x = _dev(torch, rng.random(graph.V).astype(np.float32), torch.float32)
    lab = _dev(torch, rng.permutation(graph.V).astype(np.int32), torch.int32)
    ref = torch.empty(max(rows, 1), dtype=torch.float32, device="cuda")
    ref_i = torch.empty(max(rows, 1), dtype=torch.int32, device="cuda")
    C.cg_seg_gather(seg, C.CG_OP_SUM_F32, x, ref)
    C.cg_seg_gather(seg, C.CG_OP_MIN_I32, lab, ref_i)
    both = info["staged_segments"] > 0 and info["staged_edges"] < graph.E
    for ow in (1, 4, 8, 16, 24):
        C.pr_set_gather_overlap(seg, ow)
        assert seg.info["gather_overlap"] == (ow if both else 0)
        got = torch.full_like(ref, float("nan"))
        got_i = torch.full_like(ref_i, -7)
        C.cg_seg_gather(seg, C.CG_OP_SUM_F32, x, got)
        C.cg_seg_gather(seg, C.CG_OP_MIN_I32, lab, got_i)
        assert torch.equal(got[:rows], ref[:rows]), ow
        assert torch.equal(got_i[:rows], ref_i[:rows]), ow
    C.pr_set_gather_overlap(seg, 0)
    assert seg.info["gather_overlap"] == 0
    if name in ("rmat16", "cold_hub", "ragged"):
        assert both
    if name == "rmat16":
        base, rb = P.SegmentedPageRank(graph, bounds=b).run(20)
        for ow in (4, 12):
            rank, resid = P.SegmentedPageRank(graph, bounds=b, overlap=ow).run(20)
            assert torch.equal(rank, base) and torch.equal(resid, rb)


def test_gather_overlap_rejects_bad_settings(C, torch_mod, rmat16):
    from paper_1608_01362_gb300 import pipeline as P
    graph = P.Graph(rmat16.offsets, rmat16.src, cluster_mode=0)
    b = C.pr_plan_bounds(graph.outdeg, 512, 2.0, 3000)
    pr = P.SegmentedPageRank(graph, bounds=b)
    for bad in (-1, 25, 32):
        with pytest.raises(C.CagraError, match="cached_warps"):
            C.pr_set_gather_overlap(pr.seg, bad)
    C.pr_set_gather_config(pr.seg, 512, 2, -1)
    with pytest.raises(C.CagraError, match="overlap"):
        C.pr_set_gather_overlap(pr.seg, 8)
    assert pr.info["gather_overlap"] == 0  # the previous, valid configuration stays
    C.pr_set_gather_config(pr.seg, 1024, 1, -1)
    C.pr_set_gather_overlap(pr.seg, 8)
    assert pr.info["gather_overlap"] == 8
    # the shape setter keeps the overlap request, and refuses shapes it cannot serve
    with pytest.raises(C.CagraError, match="overlap"):
        C.pr_set_gather_config(pr.seg, 512, 2, -1)
    C.pr_set_gather_config(pr.seg, 1024, 1, 4096)
    assert pr.info["gather_overlap"] == 8


def test_planned_bounds(C, torch_mod, rmat16, rmat16_oracle):
    torch = torch_mod
    from paper_1608_01362_gb300 import pipeline as P
    graph = P.Graph(rmat16.offsets, rmat16.src, cluster_mode=0)
    od = graph.outdeg.cpu().numpy()
    b = C.pr_plan_bounds(graph.outdeg, 2048, 8.0, 20000)
    # head: full 2048-vertex segments with >= 8 out-edges per vertex; then <= 20000-vertex ones
    assert b[0] == 0 and b[-1] == graph.V and np.all(np.diff(b) > 0)
    m = 0
    while m + 1 < len(b) and b[m + 1] - b[m] == 2048 and od[b[m]:b[m + 1]].sum() >= 8 * 2048:
        m += 1
    assert m >= 1
    # cold segments of <= 20000 sources; the trailing sources without out-edges
    # form one segment of their own, whatever its size
    d = np.diff(b[m:])
    assert np.all(d[:-1] <= 20000) and (d[-1] <= 20000 or od[b[-2]:].sum() == 0)
    if b[m] + 2048 <= graph.V:
        assert od[b[m]:b[m] + 2048].sum() < 8 * 2048
    pr = P.SegmentedPageRank(graph, bounds=b, threads=512, ctas_per_sm=2, table_vertices=2048)
    assert pr.info["table_vertices"] == 2048 and pr.info["staged_segments"] >= m
    rank, _ = pr.run(20)
    check_pagerank(rank.cpu().numpy(), rmat16_oracle[0], rmat16_oracle[2], what="planned bounds")
    # segment build on planned bounds is still bit-exact
    _check_segments(C, torch, graph.offsets.cpu().numpy(), graph.src.cpu().numpy(), len(b) - 1,
                    4096, bounds=b)


def test_planned_bounds_default_cold_size_from_l2(C, torch_mod, rmat16):
    """With max_global_vertices <= 0 the cold segments hold at most half of the
    L2's bytes in 4-byte values (the L2 size read from the device)."""
    import torch
    from paper_1608_01362_gb300 import pipeline as P
    graph = P.Graph(rmat16.offsets, rmat16.src, cluster_mode=0)
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    assert l2 > 0
    # no shared-memory head (threshold above any degree): only L2-sized segments
    b = C.pr_plan_bounds(graph.outdeg, -1, 1e12, -1)
    assert b[0] == 0 and b[-1] == graph.V
    assert np.all(np.diff(b) <= l2 // 8)
    # a tiny explicit size still wins; the trailing sources without out-edges
    # (the end of the clustered range) form one segment of their own
    b2 = C.pr_plan_bounds(graph.outdeg, -1, 1e12, 1000)
    od = graph.outdeg.cpu().numpy()
    end = int(np.flatnonzero(od > 0)[-1]) + 1
    assert len(b2) - 1 == -(-end // 1000) + (end < graph.V)
    assert np.all(np.diff(b2)[:-1] <= 1000) and b2[-2] == end and od[end:].sum() == 0


@pytest.mark.parametrize("table", [2048, 8192])
def test_affine_cold_segments(C, torch_mod, rmat16, rmat16_oracle, table):
    """The nested plan: the cold range cut into table-sized segments, each
    staged by one block (tables well below the capacity, so that RMAT-16 has
    many such segments).  PageRank per vertex within the bound, the integer
    gather + merge exact, and label propagation through it bit for bit."""
    torch = torch_mod
    from paper_1608_01362_gb300 import pipeline as P
    graph = P.Graph(rmat16.offsets, rmat16.src, cluster_mode=0)
    H = table
    b = P.plan_bounds(graph, 1, 24.0, max_global_vertices=H, table_vertices=table)
    pr = P.SegmentedPageRank(graph, bounds=b, table_vertices=table, affine=24.0)
    info = pr.info
    assert info["affine_segments"] >= 1 and info["affine_edges"] > 0
    assert info["staged_edges"] + info["affine_edges"] <= graph.E
    rank, _ = pr.run(20)
    check_pagerank(rank.cpu().numpy(), rmat16_oracle[0], rmat16_oracle[2], what=f"affine {table}")
    assert_gather_merge_exact(torch, C, rmat16, graph, pr.seg, f"affine {table}")
    C.pr_set_gather_affine(pr.seg, 0)  # back to the L1/L2 launch for the same segments
    assert pr.info["affine_segments"] == 0
    assert_gather_merge_exact(torch, C, rmat16, graph, pr.seg, f"affine off {table}")
    gs = graphgen.rmat(14, 8, seed=2, symmetric=True)
    gg = P.Graph(gs.offsets, gs.src, cluster_mode=0)
    lb = P.plan_bounds(gg, 1, 24.0, max_global_vertices=H, table_vertices=table)
    lp = P.LabelPropagation(gg, bounds=lb, table_vertices=table, affine=24.0)
    labels, passes, changes = lp.run()
    want, wp, wc = O.label_propagation(gs.offsets, gs.src, np.arange(gs.V, dtype=np.int32))
    assert passes == wp and np.array_equal(np.asarray(changes[:passes]), wc)
    assert np.array_equal(labels.cpu().numpy(), want)


def test_affine_rejects_bad_settings(C, torch_mod, rmat16):
    from paper_1608_01362_gb300 import pipeline as P
    graph = P.Graph(rmat16.offsets, rmat16.src, cluster_mode=0)
    H = C.pr_gather_table_capacity(1)
    pr = P.SegmentedPageRank(graph, bounds=P.plan_bounds(graph, 1, 24.0, max_global_vertices=H))
    C.pr_set_gather_config(pr.seg, 512, 2, -1)
    with pytest.raises(C.CagraError, match="1024 threads"):
        C.pr_set_gather_affine(pr.seg, 24.0)
    assert pr.info["affine_segments"] == 0
    C.pr_set_gather_config(pr.seg, 1024, 1, -1)
    C.pr_set_gather_overlap(pr.seg, 4)
    with pytest.raises(C.CagraError, match="exclude"):
        C.pr_set_gather_affine(pr.seg, 24.0)
    with pytest.raises(C.CagraError, match="head_min_avg_degree"):
        C.pr_set_gather_affine(pr.seg, -1.0)


def test_autotuner_returns_valid_choice(C, torch_mod, rmat16):
    from paper_1608_01362_gb300 import pipeline as P
    graph = P.Graph(rmat16.offsets, rmat16.src, cluster_mode=0)
    cands = P.default_candidates(uniform_k=(1, 4), shapes=((1024, 1), (512, 2)), min_deg=(16.0,),
                                 tables=(-1, 0))
    best, results = P.autotune_segments(graph, cands, iterations=2, reps=1)
    assert best in cands and len(results) == len(cands)
    assert all(r["s_per_iter"] > 0 for r in results)
