"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, brute force, invariants, printed worked examples).  CPU only."""
import json
import os

import numpy as np
import pytest

import graphgen
import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
D = O.DAMPING


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _random_graph(V, M, seed):
    rng = np.random.default_rng(seed)
    return graphgen.from_edges(V, rng.integers(0, V, M), rng.integers(0, V, M))


def _dense_transition(V, offsets, src):
    """Column-stochastic matrix built directly from the edge list: column u
    spreads 1/outdeg(u) over u's out-neighbours, dangling columns 1/V."""
    M = np.zeros((V, V))
    outdeg = np.zeros(V)
    for v in range(V):
        for u in src[offsets[v]:offsets[v + 1]]:
            outdeg[u] += 1
    for v in range(V):
        for u in src[offsets[v]:offsets[v + 1]]:
            M[v, u] += 1.0 / outdeg[u]
    for u in range(V):
        if outdeg[u] == 0:
            M[:, u] = 1.0 / V
    return M


# ---------------------------------------------------------------- PageRank

def test_cycle_is_uniform_every_iteration():
    n = 97
    g = graphgen.from_edges(n, np.arange(n), (np.arange(n) + 1) % n)
    for t in range(1, 21):
        r, _ = O.pagerank(g.offsets, g.src, iters=t)
        assert np.max(np.abs(r - 1.0 / n)) <= 4 * np.finfo(float).eps / n


def test_in_star_matches_two_variable_recurrence():
    n = 10
    N = n + 1
    # leaves 1..n -> center 0; the center has no out-edge (dangling)
    g = graphgen.from_edges(N, np.arange(1, N), np.zeros(n, dtype=int))
    x = y = 1.0 / N
    for t in range(1, 21):
        x, y = (1 - D) / N + D * y / N, (1 - D) / N + D * (n * x + y / N)
        r, _ = O.pagerank(g.offsets, g.src, iters=t)
        assert abs(r[0] - y) <= 1e-15 and np.max(np.abs(r[1:] - x)) <= 1e-15
    r, _ = O.pagerank(g.offsets, g.src, iters=400)
    assert abs(r[1] - 1.0 / (N + D * n)) < 1e-14
    assert abs(r[0] - (1 + D * n) / (N + D * n)) < 1e-14


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_rank_mass_is_one(seed):
    g = _random_graph(300, 700, seed)
    od = O.out_degree(g.offsets, g.src)
    assert (od == 0).sum() > 0  # dangling vertices present
    for t in (1, 5, 20):
        r, _ = O.pagerank(g.offsets, g.src, iters=t)
        assert abs(r.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("V,M,seed", [(8, 20, 1), (33, 90, 2), (64, 300, 3), (64, 40, 4)])
def test_dense_power_iteration(V, M, seed):
    g = _random_graph(V, M, seed)
    T = _dense_transition(V, g.offsets, g.src)
    r = np.full(V, 1.0 / V)
    for _ in range(20):
        r = (1 - D) / V + D * (T @ r)
    got, resid = O.pagerank(g.offsets, g.src, iters=20)
    assert np.max(np.abs(got - r)) < 1e-14
    assert resid.shape == (20,) and np.all(resid >= 0)


def test_fixed_point_solves_linear_system():
    V = 40
    g = _random_graph(V, 120, 7)
    T = _dense_transition(V, g.offsets, g.src)
    exact = np.linalg.solve(np.eye(V) - D * T, np.full(V, (1 - D) / V))
    got, resid = O.pagerank(g.offsets, g.src, iters=300)
    assert np.max(np.abs(got - exact)) < 1e-13
    assert resid[-1] < 1e-15 and resid[0] > resid[10] > resid[100]


# ---------------------------------------------------------------- degrees

def test_out_degree_counts_sources():
    g = _random_graph(50, 200, 11)
    assert np.array_equal(O.out_degree(g.offsets, g.src), np.bincount(g.src, minlength=50))


# ---------------------------------------------------------------- segmenting

def test_fig4_destination_sets_and_expansion_factor():
    gd = _gold("fig4_segments.json")
    e = np.array(gd["edges_src_dst"])
    g = graphgen.from_edges(gd["V"], e[:, 0], e[:, 1])
    s = O.build_segments(g.offsets, g.src, k=gd["k"], B=2)
    assert list(s.bounds) == [0, 3, 6]
    for seg_id, want in enumerate(gd["subgraph_destinations"]):
        lo, hi = s.row_base[seg_id], s.row_base[seg_id + 1]
        assert list(s.idx_map[lo:hi]) == want
    assert s.rows * gd["expansion_factor_den"] == gd["V"] * gd["expansion_factor_num"]
    # every edge of subgraph s has its source in segment s
    for seg_id, members in enumerate(gd["segments"]):
        cols = s.col[s.edge_base[seg_id]:s.edge_base[seg_id + 1]]
        assert set(cols.tolist()) <= set(members)


@pytest.mark.parametrize("k", [1, 2, 3, 8, 30, 300])
def test_expansion_factor_of_a_uniform_random_graph(k):
    """Section III-D's model of q for a uniformly sparse graph: a segment of m
    sources reaches a destination with probability 1 - (1 - p)^m, so
    E[q] = sum over segments and destinations of that probability / V
    (k (1 - (1 - p)^(V/k)) for equal segments; here with the self-loop the
    cleaned graph drops, m - 1 for a destination inside its own segment).
    The indicators are independent, so q of one directed G(V, p) sample lies
    within a few standard deviations of E[q]; counting a segment's edges
    instead of its distinct destinations (q = E/V, about 9) lies far outside
    that band up to k = 30."""
    V, p = 3000, 0.003
    rng = np.random.default_rng(21)
    adj = rng.random((V, V), dtype=np.float32) < p  # adj[u, v]: edge u -> v
    u, v = np.nonzero(adj)
    g = graphgen.from_edges(V, u, v)
    q = O.build_segments(g.offsets, g.src, k=k, B=256).q
    b = O.uniform_bounds(V, k)
    mean = var = 0.0
    for s in range(k):
        m = int(b[s + 1] - b[s])
        inside = 1.0 - (1.0 - p) ** (m - 1)   # destinations in the segment
        outside = 1.0 - (1.0 - p) ** m
        mean += m * inside + (V - m) * outside
        var += m * inside * (1 - inside) + (V - m) * outside * (1 - outside)
    mean, sd = mean / V, np.sqrt(var) / V
    assert abs(q - mean) <= 6 * sd, (q, mean, sd)
    assert q <= min(k, g.E / V)
    if k <= 30:
        assert abs(g.E / V - mean) > 20 * sd


def _brute_segments(V, offsets, src, bounds):
    """Dictionary-of-lists restatement of Algorithm 2 for tiny graphs."""
    k = len(bounds) - 1
    subs = [dict() for _ in range(k)]
    for v in range(V):
        for u in src[offsets[v]:offsets[v + 1]]:
            s = next(i for i in range(k) if bounds[i] <= u < bounds[i + 1])
            subs[s].setdefault(v, []).append(int(u))
    return subs


@pytest.mark.parametrize("V,M,k,B,seed", [(16, 40, 1, 4, 1), (16, 40, 3, 4, 2), (16, 60, 5, 3, 3),
                                          (13, 30, 4, 5, 4), (16, 10, 16, 1, 5), (7, 0, 2, 2, 6)])
def test_segments_brute_force(V, M, k, B, seed):
    g = _random_graph(V, M, seed)
    s = O.build_segments(g.offsets, g.src, k=k, B=B)
    subs = _brute_segments(V, g.offsets, g.src, s.bounds)
    for seg_id in range(k):
        rows = range(s.row_base[seg_id], s.row_base[seg_id + 1])
        want = subs[seg_id]
        assert [int(s.idx_map[i]) for i in rows] == sorted(want)
        for i in rows:
            assert s.col[s.row_ptr[i]:s.row_ptr[i + 1]].tolist() == want[int(s.idx_map[i])]
        # block indices: local row ranges of each block of B destinations
        nb = -(-V // B)
        bs = s.block_start[seg_id * (nb + 1):(seg_id + 1) * (nb + 1)]
        dst = [int(s.idx_map[i]) for i in rows]
        for b in range(nb):
            assert [x for x in dst if b * B <= x < (b + 1) * B] == dst[bs[b]:bs[b + 1]]
        assert bs[nb] == len(dst)


@pytest.mark.parametrize("k", [1, 2, 4, 7, 16])
def test_segment_invariants_rmat(k):
    g = graphgen.rmat(12, 16, seed=1)
    s = O.build_segments(g.offsets, g.src, k=k, B=256)
    assert s.edge_base[-1] == g.E and s.row_ptr[-1] == g.E
    assert np.all(np.diff(s.row_ptr) >= 1)  # no empty subgraph row
    seg_of_col = np.searchsorted(s.bounds, s.col, side="right") - 1
    seg_of_edge = np.searchsorted(s.edge_base, np.arange(g.E), side="right") - 1
    assert np.array_equal(seg_of_col, seg_of_edge)
    for seg_id in range(k):
        idx = s.idx_map[s.row_base[seg_id]:s.row_base[seg_id + 1]]
        assert np.all(np.diff(idx) > 0)
        # rows of segment s = destinations having an in-edge from segment s
        dst_of_edge = np.repeat(np.arange(g.V), np.diff(g.offsets))
        mask = (g.src >= s.bounds[seg_id]) & (g.src < s.bounds[seg_id + 1])
        assert np.array_equal(idx, np.unique(dst_of_edge[mask]))
    # q bounded by k and by the average degree (Section III-D)
    assert s.q <= k + 1e-12 and s.q <= g.E / g.V + 1e-12
    # the edges of every destination, concatenated over segments, are the row
    # of the parent CSR split stably by segment
    assert sorted(s.col.tolist()) == sorted(g.src.tolist())


def test_nonuniform_bounds_and_empty_segment():
    g = graphgen.rmat(9, 8, seed=2)
    bounds = np.array([0, 10, 10, 300, g.V], dtype=np.int64)
    s = O.build_segments(g.offsets, g.src, bounds=bounds, B=64)
    assert s.row_base[2] == s.row_base[1] and s.edge_base[2] == s.edge_base[1]
    subs = _brute_segments(g.V, g.offsets, g.src, bounds)
    assert [len(x) for x in subs] == list(np.diff(s.row_base))


# ---------------------------------------------------------------- segmented PR

def test_segmented_k1_equals_plain_bitwise():
    g = graphgen.rmat(11, 16, seed=5)
    od = O.out_degree(g.offsets, g.src)
    s = O.build_segments(g.offsets, g.src, k=1, B=128)
    a, ra = O.pagerank(g.offsets, g.src, iters=20)
    b, rb = O.pagerank_segmented(s, od, iters=20)
    assert np.array_equal(a, b) and np.array_equal(ra, rb)


@pytest.mark.parametrize("k,B", [(2, 64), (5, 1000), (16, 7), (64, 4096)])
def test_segmented_equals_plain_to_rounding(k, B):
    g = graphgen.rmat(11, 16, seed=6)
    od = O.out_degree(g.offsets, g.src)
    s = O.build_segments(g.offsets, g.src, k=k, B=B)
    a, _ = O.pagerank(g.offsets, g.src, iters=20)
    b, _ = O.pagerank_segmented(s, od, iters=20)
    assert np.sum(np.abs(a - b)) / np.sum(np.abs(a)) < 1e-14


# ---------------------------------------------------------------- clustering

def test_cluster_golden():
    gd = _gold("cluster_small.json")
    od = np.array(gd["out_degree"])
    n2o, o2n = O.cluster(od, 0)
    assert o2n.tolist() == gd["mode0_old_of_new"]
    assert np.array_equal(n2o[o2n], np.arange(len(od)))
    n2o, o2n = O.cluster(od, 1, E=gd["E"])
    assert o2n.tolist() == gd["mode1_old_of_new"]


@pytest.mark.parametrize("mode", [0, 1])
def test_cluster_order_and_relabel_isomorphism(mode):
    g = graphgen.rmat(10, 16, seed=4)
    od = O.out_degree(g.offsets, g.src)
    n2o, o2n = O.cluster(od, mode, E=g.E)
    assert np.array_equal(np.sort(o2n), np.arange(g.V))
    key = od if mode == 0 else od // max(1, g.E // g.V)
    k_new = key[o2n]
    assert np.all(np.diff(k_new) <= 0)
    same = np.diff(k_new) == 0
    assert np.all(np.diff(o2n)[same] > 0)  # ties keep the old order
    noff, nsrc = O.relabel(g.offsets, g.src, n2o, o2n)
    # edge u->v becomes n2o[u] -> n2o[v]; in-row order preserved
    for v_new in [0, 1, 2, g.V // 2, g.V - 1]:
        v_old = o2n[v_new]
        old_row = g.src[g.offsets[v_old]:g.offsets[v_old + 1]]
        assert nsrc[noff[v_new]:noff[v_new + 1]].tolist() == n2o[old_row].tolist()
    e_old = set(zip(g.src.tolist(), np.repeat(np.arange(g.V), np.diff(g.offsets)).tolist()))
    e_new = set(zip(nsrc.tolist(), np.repeat(np.arange(g.V), np.diff(noff)).tolist()))
    assert {(int(n2o[u]), int(n2o[v])) for u, v in e_old} == e_new
    # new out-degrees are the old ones, permuted
    assert np.array_equal(O.out_degree(noff, nsrc), od[o2n])
    # PageRank is equivariant under the renumbering
    a, _ = O.pagerank(g.offsets, g.src, iters=5)
    b, _ = O.pagerank(noff, nsrc, iters=5)
    assert np.max(np.abs(a[o2n] - b)) < 1e-15


# ---------------------------------------------------------------- label propagation

def test_lp_equals_connected_components():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    g = graphgen.rmat(11, 2, seed=8, symmetric=True)
    labels, passes, changes = O.label_propagation(g.offsets, g.src, np.arange(g.V, dtype=np.int32))
    A = sp.csr_matrix((np.ones(g.E), g.src, g.offsets), shape=(g.V, g.V))
    ncomp, comp = csgraph.connected_components(A, directed=False)
    rep = np.full(ncomp, g.V)
    np.minimum.at(rep, comp, np.arange(g.V))
    assert np.array_equal(labels, rep[comp])
    assert changes[-1] == 0 and np.all(changes[:-1] > 0) and ncomp > 1


def test_lp_path_needs_n_minus_1_changing_passes():
    n = 50
    a, b = np.arange(n - 1), np.arange(1, n)
    g = graphgen.from_edges(n, np.concatenate([a, b]), np.concatenate([b, a]))
    labels, passes, changes = O.label_propagation(g.offsets, g.src, np.arange(n, dtype=np.int32))
    assert passes == n and np.all(labels == 0)
    assert list(changes) == list(range(n - 1, 0, -1)) + [0]


def test_lp_single_pass_against_definition():
    g = _random_graph(40, 100, 9)
    lab = np.random.default_rng(0).permutation(40).astype(np.int32)
    out, changed = O.label_propagation_pass(g.offsets, g.src, lab)
    want = lab.copy()
    for v in range(40):
        for u in g.src[g.offsets[v]:g.offsets[v + 1]]:
            want[v] = min(want[v], lab[u])
    assert np.array_equal(out, want) and changed == int((want != lab).sum())


# ---------------------------------------------------------------- collaborative filtering

def test_cf_single_rating_golden():
    gd = _gold("cf_single_rating.json")
    uoff = np.array([0, 1]); item = np.array([0]); rate = np.array([gd["r"]], dtype=np.uint8)
    P = np.array([[gd["p"]]]); Q = np.array([[gd["q"]]])
    P2, Q2, sse = O.cf_sweep(1, 1, uoff, item, rate, uoff, np.array([0]), rate, P, Q,
                             lam=gd["lambda"], step=gd["step"])
    assert abs(P2[0, 0] - gd["p_next"]) < 1e-15 and abs(Q2[0, 0] - gd["q_next"]) < 1e-15
    assert sse == gd["sse"]


def _tiny_ratings(U=5, I=4, seed=3):
    rng = np.random.default_rng(seed)
    pairs = [(u, i) for u in range(U) for i in range(I) if rng.random() < 0.6]
    pairs += [(u, u % I) for u in range(U)]
    pairs = sorted(set(pairs))
    uoff = np.zeros(U + 1, dtype=np.int64)
    for u, _ in pairs:
        uoff[u + 1] += 1
    uoff = np.cumsum(uoff)
    item = np.array([i for _, i in pairs], dtype=np.int32)
    rate = rng.integers(1, 6, len(pairs)).astype(np.uint8)
    return U, I, uoff, item, rate


def test_cf_update_is_degree_averaged_gradient_by_finite_differences():
    U, I, uoff, item, rate = _tiny_ratings()
    ioff, iuser, irate = O.item_major(U, I, uoff, item, rate)
    K = 3
    rng = np.random.default_rng(1)
    P, Q = rng.random((U, K)), rng.random((I, K))
    lam, step = 0.05, 1e-3
    users = np.repeat(np.arange(U), np.diff(uoff))

    def data_loss(P_, Q_):
        e = rate - np.einsum("ek,ek->e", P_[users], Q_[item])
        return 0.5 * np.dot(e, e)

    P2, Q2, sse = O.cf_sweep(U, I, uoff, item, rate, ioff, iuser, irate, P, Q, lam, step)
    h = 1e-6
    du, di = np.diff(uoff), np.diff(ioff)
    for u in range(U):
        for k in range(K):
            Pp, Pm = P.copy(), P.copy()
            Pp[u, k] += h; Pm[u, k] -= h
            grad = (data_loss(Pp, Q) - data_loss(Pm, Q)) / (2 * h)
            want = P[u, k] + step * (-grad / du[u] - lam * P[u, k])
            assert abs(P2[u, k] - want) < 1e-11
    for i in range(I):
        for k in range(K):
            Qp, Qm = Q.copy(), Q.copy()
            Qp[i, k] += h; Qm[i, k] -= h
            grad = (data_loss(P, Qp) - data_loss(P, Qm)) / (2 * h)
            want = Q[i, k] + step * (-grad / di[i] - lam * Q[i, k])
            assert abs(Q2[i, k] - want) < 1e-11
    assert abs(sse - 2 * data_loss(P, Q)) < 1e-9


def test_cf_loss_decreases_for_small_step():
    U, I, uoff, item, rate = _tiny_ratings(12, 9, 5)
    ioff, iuser, irate = O.item_major(U, I, uoff, item, rate)
    rng = np.random.default_rng(2)
    P, Q = rng.random((U, 4)), rng.random((I, 4))
    last = np.inf
    for _ in range(10):
        P, Q, sse = O.cf_sweep(U, I, uoff, item, rate, ioff, iuser, irate, P, Q, 0.0, 0.05)
        assert sse <= last
        last = sse


def test_item_major_transpose():
    U, I, uoff, item, rate = _tiny_ratings(7, 5, 8)
    ioff, iuser, irate = O.item_major(U, I, uoff, item, rate)
    a = sorted(zip(np.repeat(np.arange(U), np.diff(uoff)).tolist(), item.tolist(), rate.tolist()))
    b = sorted(zip(iuser.tolist(), np.repeat(np.arange(I), np.diff(ioff)).tolist(), irate.tolist()))
    assert a == b


# ---------------------------------------------------------------- batched PPR

def test_ppr_dense_brute_force_and_mass():
    V = 30
    g = _random_graph(V, 80, 12)
    seeds = np.array([0, 7, 29, 7], dtype=np.int32)
    R = O.ppr(g.offsets, g.src, seeds, iters=20)
    # dense restatement: dangling columns send their mass back to the seed
    od = np.bincount(g.src, minlength=V).astype(float)
    A = np.zeros((V, V))
    for v in range(V):
        for u in g.src[g.offsets[v]:g.offsets[v + 1]]:
            A[v, u] += 1.0 / od[u]
    for j, s in enumerate(seeds):
        t = np.zeros(V); t[s] = 1.0
        r = t.copy()
        for _ in range(20):
            r = (1 - D) * t + D * (A @ r + t * r[od == 0].sum())
        assert np.max(np.abs(R[:, j] - r)) < 1e-14
    assert np.max(np.abs(R.sum(axis=0) - 1.0)) < 1e-12
    # columns are independent of each other
    R1 = O.ppr(g.offsets, g.src, seeds[1:2], iters=20)
    assert np.array_equal(R1[:, 0], R[:, 1])


# ---------------------------------------------------------------- generators

def test_generator_determinism_and_cleanup():
    a = graphgen.rmat(10, 16, seed=1)
    b = graphgen.rmat(10, 16, seed=1)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.src, b.src)
    c = graphgen.rmat(10, 16, seed=2)
    assert not np.array_equal(a.src, c.src)
    dst = np.repeat(np.arange(a.V), np.diff(a.offsets))
    assert np.all(a.src != dst)
    for v in range(0, a.V, 37):
        row = a.src[a.offsets[v]:a.offsets[v + 1]]
        assert np.all(np.diff(row) > 0)
    s = graphgen.rmat(9, 4, seed=3, symmetric=True)
    e = set(zip(s.src.tolist(), np.repeat(np.arange(s.V), np.diff(s.offsets)).tolist()))
    assert all((v, u) in e for (u, v) in e)


def test_bipartite_shape():
    b = graphgen.bipartite(U=2000, I=300, R=40000, seed=1)
    deg = np.diff(b.user_offsets)
    assert b.R == 40000 and deg.min() >= 1 and deg.max() <= 300
    assert b.ratings.min() >= 1 and b.ratings.max() <= 5
    for u in range(0, 2000, 97):
        row = b.items[b.user_offsets[u]:b.user_offsets[u + 1]]
        assert np.all(np.diff(row) > 0)
    pop = np.bincount(b.items, minlength=300)
    assert pop.max() > 5 * np.median(pop)  # skewed popularity


def test_rmat_quadrant_probabilities_at_every_level():
    """The RMAT recipe (Chakrabarti et al.): each edge picks, bit level by bit
    level, the quadrant (source bit, destination bit) = (0,0), (0,1), (1,0),
    (1,1) with probabilities a, b, c, d = 0.57, 0.19, 0.19, 0.05,
    independently per level.  Unpermuted, at scale 20 with one edge per
    vertex (few duplicates to drop), every level's quadrant shares are within
    0.005 of those (about ten standard deviations of a million draws)."""
    scale = 20
    g = graphgen.rmat(scale, 1, seed=3, permute=False)
    dst = np.repeat(np.arange(g.V), np.diff(g.offsets))
    want = np.array([graphgen.RMAT_A, graphgen.RMAT_B, graphgen.RMAT_C,
                     1.0 - graphgen.RMAT_A - graphgen.RMAT_B - graphgen.RMAT_C])
    assert np.allclose(want, [0.57, 0.19, 0.19, 0.05])
    for level in range(scale):
        sb = (g.src >> level) & 1
        db = (dst >> level) & 1
        share = np.bincount(2 * sb + db, minlength=4) / g.E
        assert np.all(np.abs(share - want) <= 0.005), (level, share)


def test_small_graph_batch_scales_and_determinism():
    """Graph g of the batch: scale from the first draw of stream (seed, g),
    uniform over [scale_lo, scale_hi]; the same seed gives the same batch."""
    a = graphgen.small_graph_batch(count=160, seed=1, scale_lo=5, scale_hi=8)
    b = graphgen.small_graph_batch(count=160, seed=1, scale_lo=5, scale_hi=8)
    scales = np.array([int(g.V).bit_length() - 1 for g in a])
    assert all(g.V == 1 << s for g, s in zip(a, scales))
    counts = np.bincount(scales, minlength=9)[5:]
    assert counts.sum() == 160 and counts.min() >= 20  # every scale, roughly 40 each
    for g, h in zip(a, b):
        assert np.array_equal(g.offsets, h.offsets) and np.array_equal(g.src, h.src)
    for i, s in enumerate(scales):
        d = graphgen.splitmix_draws(1, i, 2)
        assert 5 + ((int(d[0]) * 4) >> 64) == s
