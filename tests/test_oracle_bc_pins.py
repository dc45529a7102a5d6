"""Pins of the betweenness-centrality oracle (oracle.betweenness: Brandes'
algorithm from a set of sources, the BC of the paper's Table V) against
closed forms, the definition evaluated by brute force, and networkx.  CPU
only."""
import itertools

import numpy as np
import pytest

import graphgen
import oracle as O


def test_directed_path_closed_form():
    """0 -> 1 -> ... -> n-1: from source s < v every vertex after v is reached
    through v, so bc[v] = #{s in S : s < v} * (n - 1 - v)."""
    n = 40
    g = graphgen.from_edges(n, np.arange(n - 1), np.arange(1, n))
    S = [0, 3, 17, 39]
    bc, per = O.betweenness(g.offsets, g.src, S)
    want = np.array([sum(s < v for s in S) * (n - 1 - v) for v in range(n)], dtype=float)
    assert np.array_equal(bc, want)
    lev, sig, _ = per[1]
    assert np.array_equal(lev[3:], np.arange(n - 3)) and np.all(lev[:3] == -1)
    assert np.all(sig[3:] == 1.0) and np.all(sig[:3] == 0.0)


def test_undirected_star_closed_form():
    """Centre 0 joined both ways to m leaves: from a leaf, the other m - 1
    leaves are reached through the centre (delta = m - 1); from the centre,
    nothing passes through a leaf."""
    m = 25
    leaves = np.arange(1, m + 1)
    g = graphgen.from_edges(m + 1, np.concatenate([leaves, np.zeros(m, int)]),
                            np.concatenate([np.zeros(m, int), leaves]))
    S = [0, 1, 7, 19]
    bc, _ = O.betweenness(g.offsets, g.src, S)
    want = np.zeros(m + 1)
    want[0] = 3 * (m - 1)
    assert np.array_equal(bc, want)


def test_complete_graph_has_no_intermediates():
    n = 12
    src, dst = zip(*[(a, b) for a in range(n) for b in range(n) if a != b])
    g = graphgen.from_edges(n, src, dst)
    bc, per = O.betweenness(g.offsets, g.src, range(n))
    assert np.all(bc == 0.0)
    assert all(np.all(p[1] == 1.0) for p in per)


def _bfs(V, adj, s):
    dist = [-1] * V
    sig = [0] * V
    dist[s], sig[s] = 0, 1
    q = [s]
    for u in q:
        for w in adj[u]:
            if dist[w] < 0:
                dist[w] = dist[u] + 1
                q.append(w)
            if dist[w] == dist[u] + 1:
                sig[w] += sig[u]
    return dist, sig


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_brute_force_definition(seed):
    """bc[v] = sum over s in S, t != s, v not in {s, t}, t reachable, of
    sigma_st(v) / sigma_st, with sigma_st(v) = sigma_sv sigma_vt when
    d(s, v) + d(v, t) = d(s, t) (exact integer path counts)."""
    rng = np.random.default_rng(seed)
    V = 14
    M = 40
    g = graphgen.from_edges(V, rng.integers(0, V, M), rng.integers(0, V, M))
    adj = [[] for _ in range(V)]
    for v in range(V):
        for u in g.src[g.offsets[v]:g.offsets[v + 1]]:
            adj[int(u)].append(v)
    S = [0, 5, 9]
    bfs = [_bfs(V, adj, x) for x in range(V)]
    want = np.zeros(V)
    for s, t, v in itertools.product(S, range(V), range(V)):
        ds, ss = bfs[s]
        dv, sv = bfs[v]
        if t == s or v in (s, t) or ds[t] < 0 or ds[v] < 0 or dv[t] < 0:
            continue
        if ds[v] + dv[t] == ds[t]:
            want[v] += ss[v] * sv[t] / ss[t]
    bc, per = O.betweenness(g.offsets, g.src, S)
    assert np.allclose(bc, want, rtol=1e-13, atol=1e-13)
    for s, (lev, sig, _) in zip(S, per):
        assert np.array_equal(lev, np.array(bfs[s][0])) and np.array_equal(sig, bfs[s][1])


def test_matches_networkx_subset_betweenness():
    nx = pytest.importorskip("networkx")
    g = graphgen.rmat(8, 8, seed=5)
    G = nx.DiGraph()
    G.add_nodes_from(range(g.V))
    for v in range(g.V):
        for u in g.src[g.offsets[v]:g.offsets[v + 1]]:
            G.add_edge(int(u), v)
    S = [0, 1, 2, 50, 100, 200]
    want = nx.betweenness_centrality_subset(G, sources=S, targets=list(range(g.V)),
                                            normalized=False)
    bc, _ = O.betweenness(g.offsets, g.src, S)
    assert np.allclose(bc, [want[v] for v in range(g.V)], rtol=1e-12, atol=1e-12)


def test_unreached_and_source_out_of_range():
    g = graphgen.from_edges(5, [0, 1], [1, 2])
    bc, per = O.betweenness(g.offsets, g.src, [0])
    lev, sig, dl = per[0]
    assert list(lev) == [0, 1, 2, -1, -1] and list(sig) == [1, 1, 1, 0, 0]
    assert list(bc) == [0, 1, 0, 0, 0]
    with pytest.raises(ValueError):
        O.bc_source(*O.out_csr(g.offsets, g.src), 5)


def test_out_csr_is_the_transpose():
    """The counting-sort transpose equals the edge list sorted by (source,
    destination), and an in-edge CSR again when transposed back."""
    g = graphgen.rmat(10, 8, seed=7)
    oo, od = O.out_csr(g.offsets, g.src)
    dst = np.repeat(np.arange(g.V), np.diff(g.offsets))
    order = np.lexsort((dst, g.src))
    assert np.array_equal(od, dst[order])
    assert np.array_equal(oo, np.concatenate([[0], np.cumsum(np.bincount(g.src, minlength=g.V))]))
    back_off, back_src = O.out_csr(oo, od)
    assert np.array_equal(back_off, g.offsets)
    want_src = np.concatenate([np.sort(g.src[g.offsets[v]:g.offsets[v + 1]]) for v in range(g.V)])
    assert np.array_equal(back_src, want_src)
