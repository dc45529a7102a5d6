"""Collaborative filtering sweeps on the GPU (through the C ABI) against the
FP64 oracle: the item-major transpose bit for bit; every sweep entry by
entry within the oracle's rounding bound (oracle.cf_sweep_bound) from the
factors the GPU holds before it; and the drift of several sweeps from the
oracle's own trajectory within bounds derived from each storage precision.

Per sweep (the bound's derivation is in oracle.cf_sweep_bound): the GPU's
stored factors are read back (decoded to FP32, exactly what the next sweep
reads), one FP64 sweep runs from them, and every entry of the GPU's next
factors must lie within the bound of an FP32 evaluation plus the storage
rounding (BF16: 2^-8 relative; BF16 hi + lo: 2^-16).  The sum of squared
errors must lie within its bound too.

Drift over T sweeps: a sweep moves a factor by step * (g - lambda x)
(step 1e-3) and stores it back.  FP32 storage rounds it with relative error
2^-24 and the FP32 gradient sums add a few more units: after T sweeps the
factors stay within about (T + 1) * 8 * 2^-24 of the largest entry (bound
used 2e-6).  BF16 storage rounds every entry once at load and once per
sweep: |x_gpu - x_64| <= (T + 1) * 2^-8 * max|x|; two planes give
(T + 1) * 2^-16 * max|x|, plus the FP32 terms.
"""
import json
import os

import numpy as np
import pytest

import graphgen
import oracle as O

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
LAM, STEP = 0.05, 1e-3


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_1608_01362_gb300 import build, cagra
    build.build()
    cagra.load()
    return torch, cagra


def _dev(torch, a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def upload(torch, C, bp):
    """User-major CSR to the device and its item-major transpose (GPU)."""
    U, I, R = bp.U, bp.I, bp.R
    uoff = _dev(torch, bp.user_offsets, torch.int64)
    uitem = _dev(torch, bp.items, torch.int32)
    urate = _dev(torch, bp.ratings, torch.uint8)
    ioff = torch.empty(I + 1, dtype=torch.int64, device="cuda")
    iuser = torch.empty(max(R, 1), dtype=torch.int32, device="cuda")
    irate = torch.empty(max(R, 1), dtype=torch.uint8, device="cuda")
    C.cf_transpose(U, I, uoff, uitem, urate, ioff, iuser, irate)
    return uoff, uitem, urate, ioff, iuser[:R], irate[:R]


@pytest.fixture(scope="module")
def small():
    return graphgen.bipartite(U=3000, I=700, R=90_000, seed=4)


def test_transpose_bitexact(env, small):
    torch, C = env
    bp = small
    d = upload(torch, C, bp)
    ioff, iuser, irate = O.item_major(bp.U, bp.I, bp.user_offsets, bp.items, bp.ratings)
    assert np.array_equal(d[3].cpu().numpy(), ioff)
    assert np.array_equal(d[4].cpu().numpy(), iuser)
    assert np.array_equal(d[5].cpu().numpy(), irate)


def _run_both(torch, C, bp, K, precision, sweeps, seed=1):
    d = upload(torch, C, bp)
    P0, Q0 = graphgen.cf_factors(bp.U, bp.I, K, seed=seed)
    P0 = P0.astype(np.float32).astype(np.float64)  # both sides start from the FP32 values
    Q0 = Q0.astype(np.float32).astype(np.float64)
    h = C.cf_create(bp.U, bp.I, K, precision, *d)
    C.cf_set_factors(h, _dev(torch, P0, torch.float32), _dev(torch, Q0, torch.float32))
    sse = torch.zeros(sweeps, dtype=torch.float64, device="cuda")
    C.cf_sweep(h, sweeps, LAM, STEP, sse)
    Pg = torch.empty((bp.U, K), dtype=torch.float32, device="cuda")
    Qg = torch.empty((bp.I, K), dtype=torch.float32, device="cuda")
    C.cf_get_factors(h, Pg, Qg)
    ioff, iuser, irate = O.item_major(bp.U, bp.I, bp.user_offsets, bp.items, bp.ratings)
    P, Q = P0, Q0
    want_sse = []
    for _ in range(sweeps):
        P, Q, s = O.cf_sweep(bp.U, bp.I, bp.user_offsets, bp.items, bp.ratings, ioff, iuser,
                             irate, P, Q, LAM, STEP)
        want_sse.append(s)
    return (Pg.cpu().numpy().astype(np.float64), Qg.cpu().numpy().astype(np.float64),
            sse.cpu().numpy(), P, Q, np.array(want_sse))


@pytest.mark.parametrize("K", [32, 16, 64])
def test_fp32_sweeps_match_oracle(env, small, K):
    torch, C = env
    T = 10
    Pg, Qg, sse, P, Q, want = _run_both(torch, C, small, K, C.CF_FP32, T)
    assert np.max(np.abs(Pg - P)) <= 2e-6 * np.max(np.abs(P))
    assert np.max(np.abs(Qg - Q)) <= 2e-6 * np.max(np.abs(Q))
    assert np.all(np.abs(sse - want) <= 1e-5 * want)
    # the loss goes down at this step size
    assert np.all(np.diff(want) < 0) and np.all(np.diff(sse) < 0)


@pytest.mark.parametrize("precision,unit", [(1, 2.0 ** -8), (2, 2.0 ** -16)])
def test_bf16_storage_within_rounding_bound(env, small, precision, unit):
    torch, C = env
    T = 10
    Pg, Qg, sse, P, Q, want = _run_both(torch, C, small, 32, precision, T)
    slack = 2e-6  # FP32 arithmetic on top of the storage rounding
    assert np.max(np.abs(Pg - P)) <= ((T + 1) * unit + slack) * np.max(np.abs(P))
    assert np.max(np.abs(Qg - Q)) <= ((T + 1) * unit + slack) * np.max(np.abs(Q))
    # RMSE difference: |e_gpu - e_64| <= |dp . q| + |p . dq| per rating
    R = small.R
    dmax = 2 * 32 * ((T + 1) * unit + slack) * np.max(np.abs(P)) * np.max(np.abs(Q))
    assert np.all(np.abs(np.sqrt(sse / R) - np.sqrt(want / R)) <= dmax)


def test_single_rating_golden_padded(env):
    """The hand-derived one-rating sweep (K = 1), embedded in K = 16 with the
    extra dimensions zero (they stay zero: their gradient and decay are 0)."""
    torch, C = env
    with open(os.path.join(GOLD, "cf_single_rating.json")) as f:
        gd = json.load(f)
    bp = graphgen.Bipartite(1, 1, np.array([0, 1], dtype=np.int64),
                            np.array([0], dtype=np.int32), np.array([gd["r"]], dtype=np.uint8))
    d = upload(torch, C, bp)
    h = C.cf_create(1, 1, 16, C.CF_FP32, *d)
    P = torch.zeros((1, 16), dtype=torch.float32, device="cuda")
    Q = torch.zeros((1, 16), dtype=torch.float32, device="cuda")
    P[0, 0], Q[0, 0] = gd["p"], gd["q"]
    C.cf_set_factors(h, P, Q)
    sse = torch.zeros(1, dtype=torch.float64, device="cuda")
    C.cf_sweep(h, 1, gd["lambda"], gd["step"], sse)
    C.cf_get_factors(h, P, Q)
    assert abs(P[0, 0].item() - gd["p_next"]) < 1e-6 and abs(Q[0, 0].item() - gd["q_next"]) < 1e-6
    assert abs(sse.item() - gd["sse"]) < 1e-6
    assert torch.count_nonzero(P[0, 1:]).item() == 0 and torch.count_nonzero(Q[0, 1:]).item() == 0


def test_unrated_vertices_only_decay(env):
    """Users and items without ratings: x' = x (1 - step lambda)."""
    torch, C = env
    U, I = 40, 30
    pairs = [(u, (3 * u) % 20) for u in range(0, 40, 2)]  # odd users, items >= 20 unrated
    uoff = np.zeros(U + 1, dtype=np.int64)
    for u, _ in pairs:
        uoff[u + 1] += 1
    uoff = np.cumsum(uoff)
    bp = graphgen.Bipartite(U, I, uoff, np.array([i for _, i in pairs], dtype=np.int32),
                            np.full(len(pairs), 3, dtype=np.uint8))
    d = upload(torch, C, bp)
    h = C.cf_create(U, I, 32, C.CF_FP32, *d)
    P0, Q0 = graphgen.cf_factors(U, I, 32, seed=5)
    Pd, Qd = _dev(torch, P0, torch.float32), _dev(torch, Q0, torch.float32)
    C.cf_set_factors(h, Pd, Qd)
    C.cf_sweep(h, 1, LAM, STEP)
    P1, Q1 = torch.empty_like(Pd), torch.empty_like(Qd)
    C.cf_get_factors(h, P1, Q1)
    f = np.float32(1.0) - np.float32(STEP) * np.float32(LAM)
    assert np.allclose(P1.cpu().numpy()[1::2], P0.astype(np.float32)[1::2] * f, rtol=1e-6)
    assert np.allclose(Q1.cpu().numpy()[20:], Q0.astype(np.float32)[20:] * f, rtol=1e-6)


def test_sweeps_deterministic(env, small):
    torch, C = env
    a = _run_both(torch, C, small, 32, C.CF_FP32, 2)
    b = _run_both(torch, C, small, 32, C.CF_FP32, 2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])


def test_cf_errors(env, small):
    torch, C = env
    d = upload(torch, C, small)
    with pytest.raises(C.CagraError):
        C.cf_create(small.U, small.I, 24, C.CF_FP32, *d)
    with pytest.raises(C.CagraError):
        C.cf_create(small.U, small.I, 32, 3, *d)
    bad = torch.full((4,), small.I, dtype=torch.int32, device="cuda")
    uoff = torch.tensor([0, 4], dtype=torch.int64, device="cuda")
    ioff = torch.empty(small.I + 1, dtype=torch.int64, device="cuda")
    out_u = torch.empty(4, dtype=torch.int32, device="cuda")
    out_r = torch.empty(4, dtype=torch.uint8, device="cuda")
    rate = torch.ones(4, dtype=torch.uint8, device="cuda")
    with pytest.raises(C.CagraError):
        C.cf_transpose(1, small.I, uoff, bad, rate, ioff, out_u, out_r)


def test_hub_item_block_update(env):
    """An item rated by every user (40,000 ratings: more than 64 gather
    pieces, so its update runs on a whole block with a fixed-order tree)."""
    torch, C = env
    U, I = 40_000, 50
    rng = np.random.default_rng(11)
    items, offs = [], [0]
    for u in range(U):
        row = sorted({0, *rng.integers(1, I, 2).tolist()})
        items += row
        offs.append(len(items))
    bp = graphgen.Bipartite(U, I, np.array(offs, dtype=np.int64), np.array(items, dtype=np.int32),
                            rng.integers(1, 6, len(items)).astype(np.uint8))
    Pg, Qg, sse, P, Q, want = _run_both(torch, C, bp, 32, C.CF_FP32, 3)
    assert np.max(np.abs(Pg - P)) <= 2e-6 * np.max(np.abs(P))
    assert np.max(np.abs(Qg - Q)) <= 2e-6 * np.max(np.abs(Q))
    assert np.all(np.abs(sse - want) <= 1e-5 * want)


@pytest.mark.parametrize("K,precision", [(32, 0), (16, 0), (64, 0), (32, 1), (32, 2), (64, 2)])
def test_each_sweep_within_per_entry_bound(env, small, K, precision):
    torch, C = env
    bp = small
    u_store = {0: 0.0, 1: O.U_BF16, 2: O.U_BF16X2}[precision]
    d = upload(torch, C, bp)
    ioff, iuser, irate = O.item_major(bp.U, bp.I, bp.user_offsets, bp.items, bp.ratings)
    P0, Q0 = graphgen.cf_factors(bp.U, bp.I, K, seed=2)
    h = C.cf_create(bp.U, bp.I, K, precision, *d)
    C.cf_set_factors(h, _dev(torch, P0, torch.float32), _dev(torch, Q0, torch.float32))
    Pg = torch.empty((bp.U, K), dtype=torch.float32, device="cuda")
    Qg = torch.empty((bp.I, K), dtype=torch.float32, device="cuda")
    sse = torch.zeros(1, dtype=torch.float64, device="cuda")
    worst = 0.0
    for t in range(4):
        C.cf_get_factors(h, Pg, Qg)  # what the GPU's next sweep reads
        P = Pg.cpu().numpy().astype(np.float64)
        Q = Qg.cpu().numpy().astype(np.float64)
        C.cf_sweep(h, 1, LAM, STEP, sse)
        C.cf_get_factors(h, Pg, Qg)
        Pn, Qn, s64, bP, bQ, bs = O.cf_sweep_bound(bp.U, bp.I, bp.user_offsets, bp.items,
                                                   bp.ratings, ioff, iuser, irate, P, Q, LAM,
                                                   STEP, u_store=u_store)
        eP = np.abs(Pg.cpu().numpy().astype(np.float64) - Pn)
        eQ = np.abs(Qg.cpu().numpy().astype(np.float64) - Qn)
        assert np.all(eP <= bP), f"sweep {t}: {np.sum(eP > bP)} P entries outside the bound"
        assert np.all(eQ <= bQ), f"sweep {t}: {np.sum(eQ > bQ)} Q entries outside the bound"
        assert abs(float(sse.item()) - s64) <= bs
        worst = max(worst, float(np.max(eP / bP)), float(np.max(eQ / bQ)))
    assert worst > 0.0  # the GPU's rounding is seen at all (not a copy of the oracle)
