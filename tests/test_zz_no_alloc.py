"""The allocation-free plain PageRank entry point, for callers that cannot
allocate device memory at call time: its output must match the regular
plain entry point (which keeps its buffers in a handle) on two calls in a
row, and oversized inputs must be refused.  Collected last on purpose."""
import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu

TOL = 1e-6  # relative, per vertex: both paths run the same FP32 kernels and order


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


def test_noalloc_matches_plain_on_two_calls():
    torch, C, g, off, src, inv = _setup()
    V, dev = g.V, off.device
    f = lambda: torch.empty(V, dtype=torch.float32, device=dev)
    d = lambda: torch.zeros(1, dtype=torch.float64, device=dev)
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
        a, b = rn.cpu().numpy(), rp.cpu().numpy()
        assert np.max(np.abs(a - b) / np.abs(b)) <= TOL, call
        assert abs(Dn.item() - Dp.item()) <= TOL * abs(Dp.item()) + 1e-15
        assert abs(resn.item() - resp.item()) <= TOL * abs(resp.item()) + 1e-12
        rin, cin, rin_p, cin_p = rn, cn, rp, cp


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
