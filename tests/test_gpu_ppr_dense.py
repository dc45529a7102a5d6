"""The dense hub block of the batched personalised PageRank on the tensor
cores (tcgen05.mma, BF16 operands, FP32 accumulators in tensor memory).

The split is integer work: bit for bit against numpy.  The PageRank results
are compared entry by entry with the FP64 oracle's rounding bound, taken with
an accumulation unit roundoff of 2^-23: every product of a 0/1 entry and a
BF16 value is exact, and a tensor-core sum of non-negative terms may truncate
instead of rounding, which at most doubles the relative error of each
addition (the bound holds for any summation order).  Storage rounding of the
contributions as a BF16 hi + lo pair: 2^-16 (one plane: 2^-8)."""
import numpy as np
import pytest

import graphgen
import oracle as O
from parity import assert_within_bound, ppr_ref

pytestmark = pytest.mark.gpu

U_TC = 2.0 ** -23


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_1608_01362_gb300 import build, cagra, pipeline
    build.build()
    cagra.load()
    return torch, cagra, pipeline


@pytest.fixture(scope="module")
def rmat13():
    return graphgen.rmat(13, 16, seed=3)


def _seeds(g, n=64, seed=5):
    od = np.bincount(g.src, minlength=g.V)
    rng = np.random.default_rng(seed)
    hubs = list(np.argsort(-od)[:8])            # seeds inside the hub block
    rest = rng.choice(np.flatnonzero(od > 0), size=n - 8, replace=False)
    return np.asarray(hubs + list(rest), dtype=np.int32)[:n]


@pytest.mark.parametrize("h", [128, 512])
def test_split_hub_block_bitexact(env, rmat13, h):
    torch, C, P = env
    g = rmat13
    graph = P.Graph(g.offsets, g.src, cluster_mode=0)
    off, src = graph.offsets.cpu().numpy(), graph.src.cpu().numpy()
    ro = torch.empty_like(graph.offsets)
    rs = torch.empty_like(graph.src)
    bits = torch.empty(h * (h // 32), dtype=torch.int32, device="cuda")
    er = C.cg_split_hub_block(graph.offsets, graph.src, h, ro, rs, bits)
    dst = np.repeat(np.arange(graph.V), np.diff(off))
    hub = (dst < h) & (src < h)
    assert er == int((~hub).sum())
    want_off = np.concatenate([[0], np.cumsum(np.bincount(dst[~hub], minlength=graph.V))])
    assert np.array_equal(ro.cpu().numpy(), want_off)
    assert np.array_equal(rs.cpu().numpy()[:er], src[~hub])
    want_bits = np.zeros((h, h // 32), dtype=np.uint32)
    np.bitwise_or.at(want_bits, (dst[hub], src[hub] // 32),
                     (np.uint32(1) << (src[hub] % 32).astype(np.uint32)))
    assert np.array_equal(bits.cpu().numpy().view(np.uint32).reshape(h, h // 32), want_bits)


@pytest.mark.parametrize("h,k,planes", [(128, 1, 2), (512, 1, 2), (1024, 3, 2), (512, 2, 1)])
def test_dense_ppr_matches_oracle(env, rmat13, h, k, planes):
    torch, C, P = env
    g = rmat13
    graph = P.Graph(g.offsets, g.src, cluster_mode=0)
    seeds = _seeds(g)
    b = P.BatchedPPR(graph, num_segments=k, planes=planes, dense_hubs=h)
    R, _ = b.run(seeds, iterations=20)
    got = R.cpu().numpy()
    u_store = O.U_BF16X2 if planes == 2 else O.U_BF16
    want, bound = ppr_ref(g, seeds, u_store=u_store)
    bound_tc = np.stack([O.pagerank_bound(g.offsets, g.src, iters=20, seed=int(s),
                                          u_acc=U_TC, u_store=u_store)[1] for s in seeds], axis=1)
    assert np.all(bound_tc >= bound)
    assert_within_bound(got, want, bound_tc, f"dense h={h} k={k} planes={planes}")
    # the same solve without the dense block agrees within both bounds
    ref = P.BatchedPPR(graph, num_segments=k, planes=planes).run(seeds, iterations=20)[0]
    assert np.all(np.abs(got - ref.cpu().numpy()) <= bound + bound_tc)


def test_dense_ppr_deterministic_and_errors(env, rmat13):
    torch, C, P = env
    g = rmat13
    graph = P.Graph(g.offsets, g.src, cluster_mode=0)
    seeds = _seeds(g)
    b = P.BatchedPPR(graph, num_segments=1, planes=2, dense_hubs=256)
    a1 = b.run(seeds, iterations=5)[0].clone()
    a2 = b.run(seeds, iterations=5)[0]
    assert torch.equal(a1, a2)
    with pytest.raises(C.CagraError, match="attached already"):
        C.ppr_batched_attach_dense(b.ppr, 256, b.bits)
    plain = P.BatchedPPR(graph, num_segments=1, planes=2)
    with pytest.raises(C.CagraError, match="multiple of 128"):
        C.ppr_batched_attach_dense(plain.ppr, 200, b.bits)
    with pytest.raises(C.CagraError, match="multiple of 128"):
        C.cg_split_hub_block(graph.offsets, graph.src, 100, torch.empty_like(graph.offsets),
                             torch.empty_like(graph.src), b.bits)
