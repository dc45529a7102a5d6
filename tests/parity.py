"""Parity checks shared by the GPU tests.

Floating-point results are compared with the FP64 oracle element by element:
every vertex must lie within the oracle's rigorous per-vertex rounding bound
(oracle.pagerank_bound: any evaluation of the iteration in FP32 arithmetic,
with contributions stored at a given precision, in any summation order,
stays inside it), and the relative L1 error, the figure the benchmark
reports, must stay at or below its stated tolerance."""
import numpy as np

import oracle as O

TOL_L1 = 1e-5  # relative L1 of FP32 PageRank vs the FP64 oracle after 20 iterations


def rel_l1(got, want):
    got = np.asarray(got, np.float64)
    return float(np.abs(got - want).sum() / np.abs(want).sum())


def assert_within_bound(got, want, bound, what=""):
    """|got - want| <= bound at every element; on failure name the worst one."""
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    bound = np.asarray(bound, np.float64).ravel()
    err = np.abs(got - want)
    bad = ~(err <= bound)  # NaN counts as outside
    if bad.any():
        i = int(np.argmax(np.where(bad, err - np.nan_to_num(bound), -np.inf)))
        raise AssertionError(
            f"{what}: {int(bad.sum())} of {err.size} entries outside the per-element rounding "
            f"bound; worst index {i}: got {got[i]!r}, oracle {want[i]!r}, bound {bound[i]!r}")


def check_pagerank(got, want, bound, tol_l1=TOL_L1, what="pagerank"):
    """The per-vertex bound everywhere and the relative L1 tolerance."""
    assert_within_bound(got, want, bound, what)
    e = rel_l1(got, want)
    assert e <= tol_l1, f"{what}: relative L1 {e:.3e} > {tol_l1:.1e}"


def pagerank_ref(g, iters=20, u_store=0.0):
    """(rank, bound) of uniform PageRank on graph g (FP32 arithmetic)."""
    return O.pagerank_bound(g.offsets, g.src, iters=iters, u_store=u_store)


def ppr_ref(g, seeds, iters=20, u_store=0.0):
    """(R, B) [V, len(seeds)]: personalised columns and their per-entry
    bounds, FP32 arithmetic with contributions stored at u_store."""
    cols = [O.pagerank_bound(g.offsets, g.src, iters=iters, seed=int(s), u_store=u_store)
            for s in seeds]
    return (np.stack([c[0] for c in cols], axis=1), np.stack([c[1] for c in cols], axis=1))


def exact_integer_inputs(V):
    """x[u] = 1 + (u * 2654435761 mod 5): small integers, so every FP32 partial
    sum of them (below 2^24) is exact in any order."""
    return (1 + (np.arange(V, dtype=np.uint64) * np.uint64(2654435761)) % np.uint64(5)).astype(
        np.float32)


def exact_in_sums(g, x):
    """Exact sum over each vertex's in-edges of x[source] (int64)."""
    vals = np.asarray(x, np.float32)[g.src].astype(np.int64)
    cs = np.zeros(len(vals) + 1, np.int64)
    np.cumsum(vals, out=cs[1:])
    return cs[g.offsets[1:]] - cs[g.offsets[:-1]]


def assert_gather_merge_exact(torch, C, g, graph, seg, what="", want=None):
    """The segmented gather (Algorithm 3) and merge (Algorithm 4) of small
    integers equal the exact in-neighbour sums bit for bit: a dropped,
    duplicated or misplaced edge or row changes some sum by at least 1.
    want: exact_in_sums(g, exact_integer_inputs(g.V)), when already known."""
    x = exact_integer_inputs(g.V)
    if want is None:
        want = exact_in_sums(g, x)
    assert want.max(initial=0) < 2 ** 24
    xd = torch.from_numpy(x).to(graph.device)
    if graph.old_of_new is not None:
        xc = torch.empty_like(xd)
        C.cg_permute4(xd, graph.old_of_new, xc)
    else:
        xc = xd
    interm = torch.empty(max(int(seg.info["rows"]), 1), dtype=torch.float32, device=graph.device)
    C.cg_seg_gather(seg, C.CG_OP_SUM_F32, xc, interm)
    out = torch.empty(g.V, dtype=torch.float32, device=graph.device)
    C.merge(seg, C.CG_OP_SUM_F32, interm, out)
    got = graph.to_original(out).cpu().numpy()
    bad = got.astype(np.int64) != want
    assert not bad.any(), (f"{what}: {int(bad.sum())} in-neighbour sums differ; first vertex "
                           f"{int(np.flatnonzero(bad)[0])}")
