"""The allocation-free plain PageRank entry point, for callers that cannot
allocate device memory at call time (a memory budget reserved up front, a
host that lets the library touch only buffers it registered, a loop that
must not risk an allocation's synchronisation).

It runs the same kernels in the same order as the regular plain entry point
(which keeps its buffers in a handle), so on two calls in a row its output
must equal that path's bit for bit; after 20 calls it must also stay within
the FP64 oracle's per-vertex rounding bound.  It must refuse oversized
inputs, leave the device's memory use unchanged, and survive offsets that do
not rise monotonically (no fault; the next valid call is exact again).  Collected last on
purpose, so that a failure here comes after every other test has run."""
import numpy as np
import pytest

import graphgen
import oracle as O
from parity import check_pagerank

pytestmark = pytest.mark.gpu


def _setup(scale=13):
    import torch
    from paper_1608_01362_gb300 import build, cagra as C
    build.build()
    g = graphgen.rmat(scale, 16, seed=4)
    dev = torch.device("cuda")
    off = torch.as_tensor(g.offsets).to(dev)
    src = torch.as_tensor(g.src).to(dev)
    od = torch.empty(g.V, dtype=torch.int32, device=dev)
    C.cg_out_degree(src, g.V, od)
    inv = torch.empty(g.V, dtype=torch.float32, device=dev)
    C.cg_inv_outdeg(od, inv)
    return torch, C, g, off, src, inv


def test_noalloc_equals_plain_bit_for_bit_on_two_calls():
    torch, C, g, off, src, inv = _setup()
    V, dev = g.V, off.device
    f = lambda: torch.empty(V, dtype=torch.float32, device=dev)  # noqa: E731
    d = lambda: torch.zeros(1, dtype=torch.float64, device=dev)  # noqa: E731
    r0, c0, D0 = f(), f(), d()
    C.pr_init(inv, r0, c0, D0)
    plain = C.pr_plain_create(off, src)
    rin, cin = r0, c0
    Dn, Dp = D0.clone(), D0.clone()
    rin_p, cin_p = r0.clone(), c0.clone()
    for call in range(2):
        rn, cn, resn = f(), f(), d()
        C.pr_iterate_plain_noalloc(off, src, inv, rin, cin, rn, cn, 0.85, Dn, resn)
        rp, cp, resp = f(), f(), d()
        C.pr_iterate_plain(plain, inv, rin_p, cin_p, rp, cp, 0.85, 1, Dp, resp)
        torch.cuda.synchronize()
        assert torch.equal(rn, rp) and torch.equal(cn, cp), call
        assert Dn.item() == Dp.item() and resn.item() == resp.item(), call
        rin, cin, rin_p, cin_p = rn, cn, rp, cp


def test_noalloc_twenty_calls_match_the_oracle():
    torch, C, g, off, src, inv = _setup()
    V, dev = g.V, off.device
    r = [torch.empty(V, dtype=torch.float32, device=dev) for _ in range(2)]
    c = [torch.empty(V, dtype=torch.float32, device=dev) for _ in range(2)]
    D = torch.zeros(1, dtype=torch.float64, device=dev)
    C.pr_init(inv, r[0], c[0], D)
    for t in range(20):
        C.pr_iterate_plain_noalloc(off, src, inv, r[t % 2], c[t % 2], r[1 - t % 2],
                                   c[1 - t % 2], 0.85, D)
    want, bound = O.pagerank_bound(g.offsets, g.src, iters=20)
    check_pagerank(r[0].cpu().numpy(), want, bound, what="allocation-free, 20 calls")


def test_noalloc_allocates_nothing():
    """After a first call (which looks up the scratch address), further calls
    change neither PyTorch's allocated bytes nor the device's free memory."""
    torch, C, g, off, src, inv = _setup(scale=12)
    V, dev = g.V, off.device
    r = [torch.empty(V, dtype=torch.float32, device=dev) for _ in range(2)]
    c = [torch.empty(V, dtype=torch.float32, device=dev) for _ in range(2)]
    D = torch.zeros(1, dtype=torch.float64, device=dev)
    res = torch.zeros(1, dtype=torch.float64, device=dev)
    C.pr_init(inv, r[0], c[0], D)
    C.pr_iterate_plain_noalloc(off, src, inv, r[0], c[0], r[1], c[1], 0.85, D, res)
    torch.cuda.synchronize()
    alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    for t in range(4):
        C.pr_iterate_plain_noalloc(off, src, inv, r[(t + 1) % 2], c[(t + 1) % 2], r[t % 2],
                                   c[t % 2], 0.85, D, res)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_nonmonotone_offsets_stay_in_bounds():
    """Offsets that do not rise monotonically are a caller error the entry
    point cannot detect without scratch.  The gather clamps each tile's row
    and edge counts to the tile, so the call completes without a fault (its
    rank values are unspecified), and the next call with a valid CSR is again
    bit for bit the regular plain path's."""
    torch, C, g, off, src, inv = _setup(scale=10)
    V, dev = g.V, off.device
    bad = g.offsets.copy()
    bad[1:-1] = bad[1:-1][np.random.default_rng(3).permutation(V - 1)]  # shuffled row ends
    bad_off = torch.as_tensor(bad).to(dev)
    r = [torch.empty(V, dtype=torch.float32, device=dev) for _ in range(3)]
    c = [torch.empty(V, dtype=torch.float32, device=dev) for _ in range(3)]
    D = torch.zeros(1, dtype=torch.float64, device=dev)
    C.pr_init(inv, r[0], c[0], D)
    D0 = D.clone()
    C.pr_iterate_plain_noalloc(bad_off, src, inv, r[0], c[0], r[1], c[1], 0.85, D)
    torch.cuda.synchronize()  # raises if the call faulted
    D.copy_(D0)
    C.pr_iterate_plain_noalloc(off, src, inv, r[0], c[0], r[1], c[1], 0.85, D)
    plain = C.pr_plain_create(off, src)
    Dp = D0.clone()
    C.pr_iterate_plain(plain, inv, r[0], c[0], r[2], c[2], 0.85, 1, Dp)
    torch.cuda.synchronize()
    assert torch.equal(r[1], r[2]) and torch.equal(c[1], c[2])


def test_noalloc_refuses_oversized_input():
    torch, C, g, off, src, inv = _setup(scale=8)
    lim = C.pr_noalloc_limits()
    assert lim["max_vertices"] == 1 << 20 and lim["scratch_bytes"] < 16 << 20
    V = lim["max_vertices"] + 1
    dev = off.device
    big_off = torch.zeros(V + 1, dtype=torch.int64, device=dev)
    empty = torch.empty(0, dtype=torch.int32, device=dev)
    vec = torch.zeros(V, dtype=torch.float32, device=dev)
    out1, out2 = torch.zeros_like(vec), torch.zeros_like(vec)
    D = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(C.CagraError, match="exceeds the fixed scratch limit"):
        C.pr_iterate_plain_noalloc(big_off, empty, vec, vec.clone(), vec.clone(), out1, out2,
                                   0.85, D)
