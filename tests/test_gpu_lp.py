"""Label propagation through the segmented structure: every pass and the
fixed point bit-exact against the FP64-free integer oracle."""
import numpy as np
import pytest

import graphgen
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    assert torch.cuda.is_available()
    from paper_1608_01362_gb300 import build, cagra
    build.build()
    cagra.load()
    return cagra


@pytest.fixture(scope="module")
def sym16():
    return graphgen.rmat(16, 4, seed=1, symmetric=True)


def _graphs():
    out = {}
    n = 60
    a, b = np.arange(n - 1), np.arange(1, n)
    out["path"] = graphgen.from_edges(n, np.concatenate([a, b]), np.concatenate([b, a]))
    out["isolated"] = graphgen.from_edges(5, [], [])
    rng = np.random.default_rng(2)
    s, d = rng.integers(0, 3000, 2500), rng.integers(0, 3000, 2500)
    out["sparse"] = graphgen.from_edges(3000, np.concatenate([s, d]), np.concatenate([d, s]))
    return out


@pytest.mark.parametrize("cluster,k,plan", [(None, 1, None), (0, 1, None), (0, 4, None),
                                            (0, 37, None), (0, None, 8.0), (1, 3, None)])
def test_lp_passes_bitexact(C, sym16, cluster, k, plan):
    import torch
    from paper_1608_01362_gb300 import pipeline as P
    g = sym16
    graph = P.Graph(g.offsets, g.src, cluster_mode=cluster)
    bounds = C.pr_plan_bounds(graph.outdeg, 2048, plan, 20000) if plan else None
    lp = P.LabelPropagation(graph, k, bounds=bounds)
    # pass by pass, in the clustered numbering, against the oracle on the renumbered graph
    off, src = graph.offsets.cpu().numpy(), graph.src.cpu().numpy()
    lab = lp.init()
    ref = lab.cpu().numpy().copy()
    a, b = lp.labels[0], lp.labels[1]
    for p in range(6):
        changed = C.lp_iterate(lp.seg, a, b)
        ref2, ch_ref = O.label_propagation_pass(off, src, ref)
        assert np.array_equal(b.cpu().numpy(), ref2) and changed == ch_ref, p
        ref = ref2
        a, b = b, a
    # full run: labels = min original ID of each component, pass count as the oracle's
    labels, passes, changes = lp.run()
    want, wpasses, wchanges = O.label_propagation(g.offsets, g.src, np.arange(g.V, dtype=np.int32))
    assert np.array_equal(labels.cpu().numpy(), want)
    assert passes == wpasses and np.array_equal(changes, wchanges)


@pytest.mark.parametrize("name", list(_graphs().keys()))
def test_lp_special_graphs(C, name):
    from paper_1608_01362_gb300 import pipeline as P
    g = _graphs()[name]
    for k in (1, 2):
        graph = P.Graph(g.offsets, g.src, cluster_mode=0)
        labels, passes, _ = P.LabelPropagation(graph, k).run()
        want, wpasses, _ = O.label_propagation(g.offsets, g.src, np.arange(g.V, dtype=np.int32))
        assert np.array_equal(labels.cpu().numpy(), want) and passes == wpasses, (name, k)


def test_lp_rejects_alias(C, sym16):
    from paper_1608_01362_gb300 import pipeline as P
    graph = P.Graph(sym16.offsets, sym16.src, cluster_mode=None)
    lp = P.LabelPropagation(graph, 2)
    lab = lp.init()
    with pytest.raises(C.CagraError, match="alias"):
        C.lp_iterate(lp.seg, lab, lab)
