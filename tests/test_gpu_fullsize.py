"""Parity at the benchmark sizes, in the launch configurations the bench times:
RMAT-25 PageRank against the full FP64 oracle, RMAT-24 label propagation bit
for bit, 64-vector PPR on RMAT-22 (sampled columns), CF on the Netflix-shaped
ratings (two sweeps) and the 1,024-graph batch (sampled graphs).  These take a
few minutes of host time for the oracle runs."""
import os
import sys

import numpy as np
import pytest

import graphgen
import oracle as O
from parity import (assert_gather_merge_exact, assert_within_bound, check_pagerank,
                    exact_in_sums, exact_integer_inputs, ppr_ref)

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_1608_01362_gb300 import build, cagra, pipeline
    build.build()
    cagra.load()
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    return torch, cagra, pipeline


def rel_l1(got, want):
    return float(np.abs(np.asarray(got, np.float64) - want).sum() / np.abs(want).sum())


@pytest.fixture(scope="module")
def rmat25():
    """RMAT-25 and its FP64 solution: rank, per-vertex FP32 rounding bound and
    residuals after 20 iterations."""
    g = graphgen.rmat(25, 16, seed=1)
    resid = np.zeros(20)
    want, bound = O.pagerank_bound(g.offsets, g.src, iters=20, resid=resid)
    return g, want, bound, resid


def test_pagerank_rmat25_every_autotuner_plan(env, rmat25):
    """20 iterations on RMAT-25 for every plan the benchmark's autotuner can
    pick (so the timed plan is always one of these): every one of the 33.5 M
    ranks within its per-vertex rounding bound, relative L1 <= 1e-5, the
    residuals, and the gather + merge of small integers exact."""
    torch, C, P = env
    g, want, bound, want_resid = rmat25
    graph = P.Graph(g.offsets, g.src, cluster_mode=0)
    sums = exact_in_sums(g, exact_integer_inputs(g.V))
    for cand in P.default_candidates(uniform_k=(1, 2, 4, 8, 16, 32, 64)):
        pr = P.build_candidate(graph, cand)
        rank, resid = pr.run(20)
        got = rank.cpu().numpy()
        check_pagerank(got, want, bound, what=str(cand))
        assert abs(float(got.astype(np.float64).sum()) - 1.0) <= 1e-4
        r = resid.cpu().numpy()
        assert np.all(np.abs(r - want_resid) <= 1e-2 * want_resid + 2.4e-7), cand
        assert_gather_merge_exact(torch, C, g, graph, pr.seg, str(cand), want=sums)
        pr.seg.close()
        del pr, rank
    del graph
    torch.cuda.empty_cache()


def test_plain_pagerank_rmat25(env, rmat25):
    """The plain pull baseline at full size, original and clustered order."""
    torch, C, P = env
    g, want, bound, _ = rmat25
    for cluster in (None, 0):
        graph = P.Graph(g.offsets, g.src, cluster_mode=cluster)
        rank, _ = P.PlainPageRank(graph).run(20)
        check_pagerank(rank.cpu().numpy(), want, bound, what=f"plain cluster={cluster}")
        del graph, rank
    torch.cuda.empty_cache()


def test_label_propagation_rmat24_full(env):
    """Undirected RMAT-24, planned segments: final labels and pass count equal
    the oracle's exactly."""
    torch, C, P = env
    g = graphgen.rmat(24, 16, seed=1, symmetric=True)
    graph = P.Graph(g.offsets, g.src, cluster_mode=0)
    lp = P.LabelPropagation(graph, bounds=P.plan_bounds(graph, 1, 24.0))
    labels, passes, changes = lp.run()
    got = labels.cpu().numpy()
    del lp, graph
    torch.cuda.empty_cache()
    want, want_passes, want_changes = O.label_propagation(g.offsets, g.src,
                                                          np.arange(g.V, dtype=np.int32))
    assert passes == want_passes
    assert np.array_equal(np.asarray(changes[:passes]), want_changes)
    assert np.array_equal(got, want)


def test_batched_ppr_rmat22_sampled_columns(env):
    """64 vectors on RMAT-22 with the bench's seeds, at every segment count
    the bench's autotuner tries (so the timed one is among them); eight
    columns against the oracle entry by entry (per-entry rounding bound with
    BF16 hi+lo storage) and within 1.5e-4 relative L1."""
    torch, C, P = env
    import bench
    g = graphgen.rmat(22, 16, seed=1)
    graph = P.Graph(g.offsets, g.src, cluster_mode=0)
    nd = int((graph.outdeg > 0).sum().item())
    seeds = bench.ppr_seeds(g)
    assert len(set(seeds.tolist())) == 64
    cols = np.array([0, 9, 18, 27, 36, 45, 54, 63])
    want, bound = ppr_ref(g, seeds[cols], u_store=O.U_BF16X2)
    for k in (1, 2, 4, 8, 16, 32):
        b = P.BatchedPPR(graph, bounds=bench._ppr_bounds(nd, graph.V, k), planes=2)
        R, _ = b.run(seeds, 20)
        got = R[:, torch.as_tensor(cols, device=R.device)].cpu().numpy()
        assert_within_bound(got, want, bound, f"RMAT-22 64-vector PPR k={k}")
        for j in range(len(cols)):
            assert rel_l1(got[:, j], want[:, j]) <= 1.5e-4
        del b, R
        torch.cuda.empty_cache()


def test_cf_netflix_shape_two_sweeps(env):
    """The full rating graph, K = 32, FP32 and BF16 hi+lo storage: each sweep
    entry by entry within the oracle's rounding bound at sampled users and
    items (from the factors the GPU holds before it); after two sweeps the
    factors within 2e-6 (FP32) or the storage bound (BF16 hi+lo) of the
    largest FP64 entry, and the FP32 SSE within 1e-5."""
    torch, C, P = env
    bp = graphgen.bipartite(seed=1)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).cuda()  # noqa: E731
    uoff, uitem, urate = (dev(bp.user_offsets, torch.int64), dev(bp.items, torch.int32),
                          dev(bp.ratings, torch.uint8))
    ioff = torch.empty(bp.I + 1, dtype=torch.int64, device="cuda")
    iuser = torch.empty(bp.R, dtype=torch.int32, device="cuda")
    irate = torch.empty(bp.R, dtype=torch.uint8, device="cuda")
    C.cf_transpose(bp.U, bp.I, uoff, uitem, urate, ioff, iuser, irate)
    P0, Q0 = graphgen.cf_factors(bp.U, bp.I, 32, seed=1)
    P0, Q0 = P0.astype(np.float32), Q0.astype(np.float32)
    io, iu, ir = O.item_major(bp.U, bp.I, bp.user_offsets, bp.items, bp.ratings)
    Pw, Qw = P0.astype(np.float64), Q0.astype(np.float64)
    want_sse = []
    for _ in range(2):
        Pw, Qw, e = O.cf_sweep(bp.U, bp.I, bp.user_offsets, bp.items, bp.ratings, io, iu, ir, Pw,
                               Qw, 0.05, 1e-3)
        want_sse.append(e)
    want_sse = np.array(want_sse)
    # per-entry checks at sampled rows: random users, the busiest users, and
    # items from the long tail up to hubs of several hundred thousand ratings
    # (the block-per-item update path)
    rng = np.random.default_rng(11)
    udeg, ideg = np.diff(bp.user_offsets), np.diff(io)
    users = np.unique(np.concatenate([rng.choice(bp.U, 4096, replace=False),
                                      np.argsort(udeg)[-16:]]))
    by_deg = np.argsort(ideg)[::-1]
    items = np.unique(np.concatenate([by_deg[[20, 100, 1000, 5000]],
                                      rng.choice(bp.I, 60, replace=False)]))
    items = items[ideg[items] <= 1_000_000]
    for prec, tol in ((C.CF_FP32, 2e-6), (C.CF_BF16X2, 3 * 2.0 ** -16 + 2e-6)):
        h = C.cf_create(bp.U, bp.I, 32, prec, uoff, uitem, urate, ioff, iuser, irate)
        C.cf_set_factors(h, dev(P0, torch.float32), dev(Q0, torch.float32))
        sse = torch.zeros(2, dtype=torch.float64, device="cuda")
        Pg = torch.empty((bp.U, 32), dtype=torch.float32, device="cuda")
        Qg = torch.empty((bp.I, 32), dtype=torch.float32, device="cuda")
        u_store = 0.0 if prec == C.CF_FP32 else O.U_BF16X2
        for t in range(2):
            C.cf_get_factors(h, Pg, Qg)  # what this sweep reads
            Pr, Qr = Pg.cpu().numpy().astype(np.float64), Qg.cpu().numpy().astype(np.float64)
            C.cf_sweep(h, 1, 0.05, 1e-3, sse[t:t + 1])
            C.cf_get_factors(h, Pg, Qg)
            Pn, Qn, _, bP, bQ, _ = O.cf_sweep_bound(bp.U, bp.I, bp.user_offsets, bp.items,
                                                    bp.ratings, io, iu, ir, Pr, Qr, 0.05, 1e-3,
                                                    u_store=u_store, users=users, items=items)
            eP = np.abs(Pg.cpu().numpy()[users].astype(np.float64) - Pn[users])
            eQ = np.abs(Qg.cpu().numpy()[items].astype(np.float64) - Qn[items])
            assert np.all(eP <= bP), f"sweep {t}: {np.sum(eP > bP)} sampled P entries outside"
            assert np.all(eQ <= bQ), f"sweep {t}: {np.sum(eQ > bQ)} sampled Q entries outside"
        # drift of the two sweeps from the oracle's own trajectory
        assert np.max(np.abs(Pg.cpu().numpy() - Pw)) <= tol * np.max(np.abs(Pw))
        assert np.max(np.abs(Qg.cpu().numpy() - Qw)) <= tol * np.max(np.abs(Qw))
        if prec == C.CF_FP32:
            assert np.all(np.abs(sse.cpu().numpy() - want_sse) <= 1e-5 * want_sse)
        del h


def test_batched_1024_graphs_sampled(env):
    """The 1,024-graph batch in one launch; 32 graphs against the oracle."""
    torch, C, P = env
    gs = graphgen.small_graph_batch(count=1024, seed=1, scale_lo=8, scale_hi=15)
    bpr = P.BatchedPageRank(gs, threads=512)
    rank = bpr.run(20).cpu().numpy()
    for i in range(0, 1024, 32):
        want, bound = O.pagerank_bound(gs[i].offsets, gs[i].src, iters=20)
        check_pagerank(rank[bpr.vbase[i]:bpr.vbase[i + 1]], want, bound, what=f"graph {i}")


def test_betweenness_rmat25_two_sources(env, rmat25):
    """Betweenness centrality on RMAT-25 (clustered) from the bench's first two
    sources: per source the levels and path counts equal the oracle's bit for
    bit and the dependencies lie within the FP64 bound of tests/test_gpu_bc.py."""
    torch, C, P = env
    import bench
    g = rmat25[0]
    S = bench.ppr_seeds(g, n=12)[:2]
    graph = P.Graph(g.offsets, g.src, cluster_mode=0)
    bc = P.Betweenness(graph)
    out_off, out_dst = O.out_csr(g.offsets, g.src)
    maxdeg = int(np.diff(out_off).max())
    for s in S:
        lev, sig, dl, depth = O.bc_source(out_off, out_dst, int(s))
        bc.run([int(s)])
        glev, gsig, gdl, info = bc.source_state()
        assert info["depth"] == depth
        assert np.array_equal(glev.cpu().numpy(), lev)
        assert sig.max() < 2.0 ** 53
        assert np.array_equal(gsig.cpu().numpy(), sig)
        tol = 2.0 * depth * (maxdeg + 8) * 2.0 ** -53
        assert np.all(np.abs(gdl.cpu().numpy() - dl) <= tol * dl + 1e-300)
    del bc, graph
    torch.cuda.empty_cache()
