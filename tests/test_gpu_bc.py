"""Betweenness centrality on the GPU (through the C ABI) against the FP64
Brandes oracle: the transpose bit for bit; per source the BFS levels and the
shortest-path counts sigma bit for bit (integers, exact in FP64 in any order
below 2^53); the centralities within the FP64 bound below, with the pull and
push directions and with and without clustering.

Tolerance.  delta[u] = sigma[u] * sum_w (1 + delta[w]) / sigma[w] over the
out-neighbours one level deeper: every term is positive, so each level adds at
most (deg(u) + 3) roundings of relative size 2^-53 to the relative error it
inherits (the GPU's sum in its own order, the oracle's in CSR order, plus the
division and products), and summing positive dependencies over sources adds
no more than the largest.  Hence, per vertex,
    |bc_gpu - bc_64| <= 2 * depth * (max_degree + 8) * 2^-53 * bc_64."""
import numpy as np
import pytest

import graphgen
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_1608_01362_gb300 import build, cagra, pipeline
    build.build()
    cagra.load()
    return torch, cagra, pipeline


def _graphs():
    rng = np.random.default_rng(11)
    n = 300
    leaves = np.arange(1, 41)
    out = {
        "path": graphgen.from_edges(n, np.arange(n - 1), np.arange(1, n)),
        "star": graphgen.from_edges(41, np.concatenate([leaves, np.zeros(40, int)]),
                                    np.concatenate([np.zeros(40, int), leaves])),
        "complete": graphgen.from_edges(
            20, *zip(*[(a, b) for a in range(20) for b in range(20) if a != b])),
        "ragged": graphgen.from_edges(500, rng.integers(0, 500, 3000),
                                      (rng.integers(0, 500, 3000) ** 2) % 500),
        "rmat12": graphgen.rmat(12, 16, seed=3),
        "rmat12_sym": graphgen.rmat(12, 8, seed=4, symmetric=True),
    }
    return out


GRAPHS = _graphs()


def _sources(g, n=6, seed=1):
    od = np.bincount(g.src, minlength=g.V)
    rng = np.random.default_rng(seed)
    picks = [int(np.argmax(od))]
    cand = np.flatnonzero(od > 0)
    picks += [int(x) for x in rng.choice(cand, size=min(n - 2, cand.size), replace=False)]
    zero = np.flatnonzero(od == 0)
    if zero.size:
        picks.append(int(zero[0]))  # a source with no out-edges
    return picks


def _tol(g, depth):
    return 2.0 * depth * (np.diff(O.out_csr(g.offsets, g.src)[0]).max(initial=0) + 8) * 2.0 ** -53


def test_transpose_bitexact(env):
    torch, C, P = env
    for name, g in GRAPHS.items():
        off = torch.as_tensor(g.offsets).cuda()
        src = torch.as_tensor(g.src).cuda()
        oo = torch.empty_like(off)
        od = torch.empty_like(src)
        C.cg_transpose_csr(off, src, oo, od)
        wo, wd = O.out_csr(g.offsets, g.src)
        assert np.array_equal(oo.cpu().numpy(), wo) and np.array_equal(od.cpu().numpy(), wd), name


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("cluster", [None, 0])
@pytest.mark.parametrize("alpha", [0.0, 16.0, 1e30])
def test_bc_matches_oracle(env, name, cluster, alpha):
    torch, C, P = env
    g = GRAPHS[name]
    graph = P.Graph(g.offsets, g.src, cluster_mode=cluster)
    bc = P.Betweenness(graph, alpha=alpha)
    S = _sources(g)
    want, per = O.betweenness(g.offsets, g.src, S)
    depth = 1
    for s, (lev, sig, dl) in zip(S, per):
        bc.run([s])
        glev, gsig, gdl, info = bc.source_state()
        assert np.array_equal(glev.cpu().numpy(), lev), (name, s)
        assert sig.max() < 2.0 ** 53
        assert np.array_equal(gsig.cpu().numpy(), sig), (name, s)
        assert info["depth"] == lev.max() + 1
        if alpha == 0.0:
            assert info["pull_levels"] == 0
        depth = max(depth, info["depth"])
        tol = _tol(g, info["depth"])
        got_d = gdl.cpu().numpy()
        assert np.all(np.abs(got_d - dl) <= tol * dl + 1e-300), (name, s)
    got = bc.run(S).cpu().numpy()
    tol = _tol(g, depth)
    assert np.all(np.abs(got - want) <= tol * want + 1e-300), name


def test_bc_closed_forms(env):
    torch, C, P = env
    n = 300
    g = GRAPHS["path"]
    bc = P.Betweenness(P.Graph(g.offsets, g.src, cluster_mode=0))
    S = [0, 3, 100, 299]
    got = bc.run(S).cpu().numpy()
    want = np.array([sum(s < v for s in S) * (n - 1 - v) for v in range(n)], dtype=float)
    assert np.array_equal(got, want)
    g = GRAPHS["complete"]
    assert np.all(P.Betweenness(P.Graph(g.offsets, g.src)).run(range(20)).cpu().numpy() == 0.0)


def test_bc_accumulates_and_is_deterministic(env):
    torch, C, P = env
    g = GRAPHS["rmat12"]
    graph = P.Graph(g.offsets, g.src, cluster_mode=0)
    bc = P.Betweenness(graph)
    S = _sources(g)
    a = bc.run(S).clone()
    b = bc.run(S)
    assert torch.equal(a, b)
    acc = torch.zeros(g.V, dtype=torch.float64, device="cuda")
    for s in S:  # one source per call adds up to the whole set (same order)
        C.bc_run(bc.h, [graph.to_clustered_id(s)], acc)
    assert torch.equal(bc.to_original8(acc), a)


def test_bc_errors(env):
    torch, C, P = env
    g = GRAPHS["ragged"]
    graph = P.Graph(g.offsets, g.src, cluster_mode=None)
    bc = P.Betweenness(graph)
    out = torch.zeros(g.V, dtype=torch.float64, device="cuda")
    with pytest.raises(C.CagraError, match="outside"):
        C.bc_run(bc.h, [g.V], out)
    with pytest.raises(C.CagraError, match="no source"):
        C.bc_source_state(P.Betweenness(graph).h)
    with pytest.raises(C.CagraError, match="alpha"):
        C.bc_set_direction(bc.h, -1.0)
    bad = torch.as_tensor(np.array([0, 2, 1, 3])).cuda()
    with pytest.raises(C.CagraError, match="INVALID_ARG"):
        C.cg_transpose_csr(bad, torch.zeros(3, dtype=torch.int32, device="cuda"),
                           torch.empty_like(bad), torch.empty(3, dtype=torch.int32, device="cuda"))
