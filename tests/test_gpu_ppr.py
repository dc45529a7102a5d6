"""Personalised PageRank on the GPU (through the C ABI) against the FP64
oracle: one vector through the segmented PageRank path, and 64 vectors at once
through the batched SpMM-form gather with BF16 hi+lo (or hi-only) storage.

Tolerances.  One vector is FP32 throughout: the same 1e-5 relative L1 as
uniform PageRank.  The batched form stores the contributions C = R / outdeg
in BF16 planes (8 significant bits, unit roundoff u = 2^-8): two planes keep
|c - (hi + lo)| <= 2^-8 |c - hi| <= 2^-16 |c|, one plane |c - hi| <= 2^-8 |c|.
The iteration map R -> d A (R / outdeg) + teleport, with the dangling mass
returned to the seed, is a contraction by d in the L1 norm, and each column
of R has L1 norm 1, so the storage error of one iteration (at most d u) adds
up to at most u d / (1 - d) = 5.67 u after any number of iterations, plus
the FP32 sums (below 1e-6 at these degrees):
    two planes:  5.67 * 2^-16 = 8.6e-5   -> bound used 1.5e-4
    one plane:   5.67 * 2^-8  = 2.2e-2   -> bound used 3e-2
"""
import numpy as np
import pytest

import graphgen
import oracle as O
from parity import assert_within_bound, ppr_ref

pytestmark = pytest.mark.gpu

TOL_SINGLE = 1e-5
TOL_PLANES = {2: 1.5e-4, 1: 3e-2}
# relative rounding of a stored contribution: BF16 hi + lo pair, BF16 alone; the
# per-entry bounds (oracle.pagerank_bound) add it to the FP32 arithmetic's
U_STORE = {2: O.U_BF16X2, 1: O.U_BF16}
COLS = 64


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_1608_01362_gb300 import build, cagra, pipeline
    build.build()
    cagra.load()
    return torch, cagra, pipeline


def col_rel_l1(got, want):
    """Per-column relative L1 of got [V, J] against want [V, J]."""
    got = np.asarray(got, np.float64)
    return np.sum(np.abs(got - want), axis=0) / np.sum(np.abs(want), axis=0)


def mixed_seeds(g, n=COLS, seed=7):
    """Seeds covering the method's cases: hubs, dangling vertices (no
    out-edges), vertices without in-edges, repeats, and random draws."""
    od = O.out_degree(g.offsets, g.src)
    indeg = np.diff(g.offsets)
    rng = np.random.default_rng(seed)
    picks = [int(np.argmax(od))]
    for mask in (od == 0, indeg == 0, (od > 0) & (indeg > 0)):
        idx = np.flatnonzero(mask)
        if idx.size:
            picks += [int(x) for x in rng.choice(idx, size=min(4, idx.size), replace=False)]
    picks += [picks[0], picks[-1]]  # repeats
    while len(picks) < n:
        picks.append(int(rng.integers(0, g.V)))
    return np.asarray(picks[:n], dtype=np.int32)


@pytest.fixture(scope="module")
def rmat13():
    return graphgen.rmat(13, 16, seed=3)


# ------------------------------------------------------------------ one vector

@pytest.mark.parametrize("k", [1, 4])
def test_single_vector_ppr(env, rmat13, k):
    torch, C, P = env
    g = rmat13
    G = P.Graph(g.offsets, g.src, cluster_mode=0)
    pr = P.SegmentedPageRank(G, num_segments=k)
    seeds = mixed_seeds(g, n=6)
    want, bound = ppr_ref(g, seeds)
    for j, s in enumerate(seeds):
        rank, resid = pr.run_ppr(int(s), iterations=20)
        assert_within_bound(rank.cpu().numpy(), want[:, j], bound[:, j], f"seed {int(s)} k={k}")
        err = col_rel_l1(rank.cpu().numpy()[:, None], want[:, j:j + 1])[0]
        assert err <= TOL_SINGLE, (int(s), err)
        assert np.all(np.isfinite(resid.cpu().numpy()))


def test_single_vector_seed_out_of_range(env, rmat13):
    torch, C, P = env
    G = P.Graph(rmat13.offsets, rmat13.src, cluster_mode=None)
    pr = P.SegmentedPageRank(G, num_segments=2)
    with pytest.raises(C.CagraError):
        C.pr_iterate_ppr(pr.seg, G.inv, pr.rank[0], pr.contrib[0], pr.rank[1], pr.contrib[1],
                         0.85, 1, G.V, pr.dangling)


# ------------------------------------------------------------------ batched (64)

@pytest.mark.parametrize("planes", [2, 1])
@pytest.mark.parametrize("k", [1, 3, 16])
def test_batched_ppr_matches_oracle(env, rmat13, planes, k):
    torch, C, P = env
    g = rmat13
    G = P.Graph(g.offsets, g.src, cluster_mode=0)
    b = P.BatchedPPR(G, num_segments=k, planes=planes)
    seeds = mixed_seeds(g)
    R, resid = b.run(seeds, iterations=20)
    want, bound = ppr_ref(g, seeds, u_store=U_STORE[planes])
    assert_within_bound(R.cpu().numpy(), want, bound, f"planes={planes} k={k}")
    err = col_rel_l1(R.cpu().numpy(), want)
    assert err.max() <= TOL_PLANES[planes], (planes, k, err.max(), int(np.argmax(err)))
    # the columns of a PPR matrix are probability vectors
    sums = R.double().sum(0).cpu().numpy()
    assert np.all(np.abs(sums - 1.0) <= 20 * TOL_PLANES[planes])


def test_batched_ppr_unclustered_plan_bounds(env):
    """Unclustered numbering and the GPU's own segment plan."""
    torch, C, P = env
    g = graphgen.rmat(14, 8, seed=11)
    G = P.Graph(g.offsets, g.src, cluster_mode=None)
    bounds = P.plan_bounds(G, min_avg_degree=4.0, max_global_vertices=1 << 12)
    b = P.BatchedPPR(G, bounds=bounds, planes=2)
    seeds = mixed_seeds(g, seed=3)
    R, _ = b.run(seeds, iterations=12)
    want, bound = ppr_ref(g, seeds, iters=12, u_store=U_STORE[2])
    assert_within_bound(R.cpu().numpy(), want, bound, "unclustered planned bounds")
    assert col_rel_l1(R.cpu().numpy(), want).max() <= TOL_PLANES[2]


def _special():
    out = {}
    out["single"] = graphgen.from_edges(1, [], [])
    out["two_isolated"] = graphgen.from_edges(2, [], [])
    n = 5000  # in-star: one destination row of 5000 edges (a run of 40 carries)
    out["in_star"] = graphgen.from_edges(n + 1, np.arange(1, n + 1), np.zeros(n, dtype=int))
    out["out_star"] = graphgen.from_edges(n + 1, np.zeros(n, dtype=int), np.arange(1, n + 1))
    m = 3000
    out["cycle"] = graphgen.from_edges(m, np.arange(m), (np.arange(m) + 1) % m)
    rng = np.random.default_rng(5)
    out["ragged"] = graphgen.from_edges(777, rng.integers(0, 777, 5000),
                                        (rng.integers(0, 777, 5000) ** 2) % 777)
    return out


@pytest.mark.parametrize("name", list(_special().keys()))
@pytest.mark.parametrize("k", [1, 2])
def test_batched_ppr_special_graphs(env, name, k):
    torch, C, P = env
    g = _special()[name]
    G = P.Graph(g.offsets, g.src, cluster_mode=0)
    b = P.BatchedPPR(G, num_segments=min(k, g.V), planes=2)
    rng = np.random.default_rng(1)
    seeds = rng.integers(0, g.V, COLS).astype(np.int32)
    seeds[0] = 0
    R, _ = b.run(seeds, iterations=20)
    want, bound = ppr_ref(g, seeds, u_store=U_STORE[2])
    assert_within_bound(R.cpu().numpy(), want, bound, name)
    assert col_rel_l1(R.cpu().numpy(), want).max() <= TOL_PLANES[2], name


def test_batched_ppr_larger_sampled(env):
    """Scale 17 (many gather chunks per segment, many merge tasks); the
    oracle computes 8 of the 64 columns."""
    torch, C, P = env
    g = graphgen.rmat(17, 16, seed=2)
    G = P.Graph(g.offsets, g.src, cluster_mode=0)
    b = P.BatchedPPR(G, num_segments=8, planes=2)
    seeds = mixed_seeds(g, seed=9)
    R, _ = b.run(seeds, iterations=20)
    cols = np.array([0, 1, 5, 9, 13, 21, 40, 63])
    want, bound = ppr_ref(g, seeds[cols], u_store=U_STORE[2])
    assert_within_bound(R.cpu().numpy()[:, cols], want, bound, "scale 17")
    assert col_rel_l1(R.cpu().numpy()[:, cols], want).max() <= TOL_PLANES[2]


def test_batched_residual_and_determinism(env, rmat13):
    """resid[j] = sum_v |R_T - R_{T-1}| (R_{T-1} from a fresh run of T-1
    iterations, which takes the same arithmetic path) up to the FP32 terms:
    each |r - r_old| is rounded in FP32 and summed in FP32 over at most 16
    destinations before the FP64 reduction, a relative error below
    17 * 2^-24 = 1.0e-6 (bound used 2e-6).  Repeated runs are bit-identical."""
    torch, C, P = env
    g = rmat13
    G = P.Graph(g.offsets, g.src, cluster_mode=0)
    b = P.BatchedPPR(G, num_segments=4, planes=2)
    seeds = mixed_seeds(g)
    R7, res7 = b.run(seeds, iterations=7)
    R7 = R7.clone()
    res7 = res7.cpu().numpy().copy()
    R6, _ = b.run(seeds, iterations=6)
    want = np.abs(R7.cpu().numpy().astype(np.float64) - R6.cpu().numpy()).sum(0)
    assert np.allclose(res7, want, rtol=2e-6, atol=1e-12)
    R7b, res7b = b.run(seeds, iterations=7)
    assert torch.equal(R7, R7b)
    assert np.array_equal(res7, res7b.cpu().numpy())


def test_batched_phases_equal_iterate(env, rmat13):
    torch, C, P = env
    g = rmat13
    G = P.Graph(g.offsets, g.src, cluster_mode=0)
    b = P.BatchedPPR(G, num_segments=3, planes=2)
    seeds = mixed_seeds(g)
    b.init(seeds)
    C.ppr_batched_iterate(b.ppr, G.inv, 0.85, 3, b.rank)
    want = b.rank.clone()
    b.init(seeds)
    out = torch.empty_like(b.rank)
    for t in range(3):
        for ph in (1, 2, 4):
            C.ppr_batched_step(b.ppr, G.inv, 0.85, ph, rank_out=out if ph == 4 else None)
    assert torch.equal(out, want)


def test_batched_errors(env, rmat13):
    torch, C, P = env
    G = P.Graph(rmat13.offsets, rmat13.src, cluster_mode=None)
    seg = C.pr_build_segments(G.offsets, G.src, 2)
    with pytest.raises(C.CagraError):
        C.ppr_batched_create(seg, 3)
    b = C.ppr_batched_create(seg, 2)
    with pytest.raises(C.CagraError):  # iterate before init
        C.ppr_batched_iterate(b, G.inv, 0.85, 1)
    bad = np.zeros(COLS, dtype=np.int32)
    bad[5] = G.V
    with pytest.raises(C.CagraError):
        C.ppr_batched_init(b, G.inv, bad)
    C.ppr_batched_init(b, G.inv, np.zeros(COLS, dtype=np.int32))
    resid = torch.zeros(COLS, dtype=torch.float64, device="cuda")
    with pytest.raises(C.CagraError):  # residual needs two iterations
        C.ppr_batched_iterate(b, G.inv, 0.85, 1, None, resid)


def test_batched_column_matches_single_vector_run(env, rmat13):
    """Each column of the batched solve is the one-vector personalised
    PageRank of its seed (same graph, same segments), within the storage bound."""
    torch, C, P = env
    g = rmat13
    G = P.Graph(g.offsets, g.src, cluster_mode=0)
    b = P.BatchedPPR(G, num_segments=4, planes=2)
    seeds = mixed_seeds(g)
    R, _ = b.run(seeds, iterations=20)
    R = R.cpu().numpy()
    pr = P.SegmentedPageRank(G, num_segments=4)
    for j in (0, 3, 17, 63):
        r1, _ = pr.run_ppr(int(seeds[j]), iterations=20)
        r1 = r1.cpu().numpy().astype(np.float64)
        assert np.sum(np.abs(R[:, j] - r1)) / np.sum(np.abs(r1)) <= TOL_PLANES[2] + TOL_SINGLE


def test_batched_columns_are_independent(env, rmat13):
    """Permuting the seeds permutes the columns bit for bit: a column's
    arithmetic never involves another column."""
    torch, C, P = env
    g = rmat13
    G = P.Graph(g.offsets, g.src, cluster_mode=0)
    b = P.BatchedPPR(G, num_segments=3, planes=2)
    seeds = mixed_seeds(g)
    R1, res1 = b.run(seeds, iterations=9)
    R1, res1 = R1.clone(), res1.clone()
    perm = np.random.default_rng(4).permutation(COLS)
    R2, res2 = b.run(seeds[perm], iterations=9)
    assert torch.equal(R2, R1[:, torch.as_tensor(perm, device="cuda")])
    assert torch.equal(res2, res1[torch.as_tensor(perm, device="cuda")])
