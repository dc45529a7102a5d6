"""Pins of the oracle's per-entry rounding bound of a collaborative-filtering
sweep (oracle.cf_sweep_bound; the CF application of Section VI, one Jacobi
gradient step over the rating graph).

The bound claims: an evaluation of the sweep in FP32 from the same factors,
summing each dot product and each vertex's gradient in any order, lands
within bound[v, k] of the FP64 sweep at every entry, and within u_store more
once it stores x' as BF16 or a BF16 hi + lo pair; its sum of squared errors
lands within bound_sse.  These tests evaluate the sweep in numpy FP32 in
several orders and storage formats and check the claim entry by entry, check
that the bound is not vacuous (it is far below a sweep's own movement and an
actual evaluation comes within a small factor of it), and that it fails
planted mistakes in an evaluation (a dropped lambda term, a dropped rating,
a flipped error sign, the wrong factor in the gradient).  CPU only."""
import numpy as np
import pytest

import graphgen
import oracle as O

LAM, STEP = 0.05, 1e-3


def _bf16(x):
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _hilo(x):
    x = np.asarray(x, np.float32)
    h = _bf16(x)
    return (h + _bf16((x - h).astype(np.float32))).astype(np.float32)


def _seq_rows(off, vals, reverse=False):
    """Per-row FP32 sums of vals (rows x K) left to right (or right to left)."""
    deg = np.diff(off)
    acc = np.zeros((len(deg),) + vals.shape[1:], np.float32)
    for j in range(int(deg.max(initial=0))):
        m = deg > j
        pos = off[:-1][m] + (deg[m] - 1 - j if reverse else j)
        acc[m] = (acc[m] + vals[pos]).astype(np.float32)
    return acc


def _side32(off, nbr, val, X, Y, order, mistake=None):
    """One side of the sweep in FP32: x + step (sum e y / deg - lambda x)."""
    off = np.asarray(off, np.int64)
    deg = np.diff(off)
    rows = np.repeat(np.arange(len(deg)), deg)
    Yr = Y[nbr]
    prod = (X[rows] * Yr).astype(np.float32)
    K = X.shape[1]
    if order == "pairwise":
        dot = prod.sum(axis=1, dtype=np.float32)
    else:
        dot = np.zeros(len(rows), np.float32)
        for k in (range(K - 1, -1, -1) if order == "reverse" else range(K)):
            dot = (dot + prod[:, k]).astype(np.float32)
    e = (val.astype(np.float32) - dot).astype(np.float32)
    if mistake == "sign":
        e = -e
    terms = (e[:, None] * (X[rows] if mistake == "factor" else Yr)).astype(np.float32)
    if mistake == "drop":  # the first rating of every vertex of degree >= 2
        first = off[:-1][deg >= 2]
        terms[first] = 0.0
    g = _seq_rows(off, terms, reverse=(order == "reverse"))
    inv = np.where(deg > 0, np.float32(1.0) / np.maximum(deg, 1).astype(np.float32),
                   np.float32(0.0)).astype(np.float32)
    a = (g * inv[:, None]).astype(np.float32)
    b = (np.float32(LAM) * X).astype(np.float32)
    c = a if mistake == "lambda" else (a - b).astype(np.float32)
    d = (np.float32(STEP) * c).astype(np.float32)
    x = (X + d).astype(np.float32)
    sse = _seq_rows(off, (e * e).astype(np.float32)[:, None])[:, 0]
    return x, sse


def _sweep32(bp, tr, P, Q, order="forward", store=None, mistake=None):
    ioff, iuser, irate = tr
    P32, Q32 = P.astype(np.float32), Q.astype(np.float32)
    Pn, sse_u = _side32(bp.user_offsets, bp.items, bp.ratings, P32, Q32, order, mistake)
    Qn, _ = _side32(ioff, iuser, irate, Q32, P32, order, mistake)
    if store is not None:
        Pn, Qn = store(Pn), store(Qn)
    return Pn.astype(np.float64), Qn.astype(np.float64), float(np.sum(sse_u.astype(np.float64)))


@pytest.fixture(scope="module")
def case():
    bp = graphgen.bipartite(U=700, I=160, R=12_000, seed=9)
    tr = O.item_major(bp.U, bp.I, bp.user_offsets, bp.items, bp.ratings)
    P, Q = graphgen.cf_factors(bp.U, bp.I, 32, seed=3)
    # the factors an FP32 evaluation reads: FP32 values
    return bp, tr, P.astype(np.float32).astype(np.float64), Q.astype(np.float32).astype(np.float64)


def _bound(case, u_store=0.0):
    bp, tr, P, Q = case
    return O.cf_sweep_bound(bp.U, bp.I, bp.user_offsets, bp.items, bp.ratings, *tr, P, Q, LAM,
                            STEP, u_store=u_store)


@pytest.mark.parametrize("order", ["forward", "reverse", "pairwise"])
def test_fp32_sweep_within_bound(case, order):
    bp, tr, P, Q = case
    Pn, Qn, sse, bP, bQ, bs = _bound(case)
    P32, Q32, s32 = _sweep32(bp, tr, P, Q, order)
    assert np.all(np.abs(P32 - Pn) <= bP)
    assert np.all(np.abs(Q32 - Qn) <= bQ)
    assert abs(s32 - sse) <= bs
    # not vacuous: the FP32 evaluation uses a visible share of the bound
    assert max(np.max(np.abs(P32 - Pn) / bP), np.max(np.abs(Q32 - Qn) / bQ)) > 0.05


@pytest.mark.parametrize("store,u_store", [(_bf16, O.U_BF16), (_hilo, O.U_BF16X2)])
def test_stored_sweep_within_bound(case, store, u_store):
    bp, tr, P, Q = case
    Pn, Qn, sse, bP, bQ, bs = _bound(case, u_store)
    P32, Q32, _ = _sweep32(bp, tr, P, Q, "forward", store)
    assert np.all(np.abs(P32 - Pn) <= bP)
    assert np.all(np.abs(Q32 - Qn) <= bQ)
    assert max(np.max(np.abs(P32 - Pn) / bP), np.max(np.abs(Q32 - Qn) / bQ)) > 0.05


def test_fp32_bound_far_below_a_sweeps_movement(case):
    """An FP32 bound that is a tiny fraction of how far one sweep moves a
    factor: a per-entry check at this bound sees a changed update."""
    bp, tr, P, Q = case
    Pn, Qn, _, bP, bQ, _ = _bound(case)
    move = np.concatenate([np.abs(Pn - P).ravel(), np.abs(Qn - Q).ravel()])
    b = np.concatenate([bP.ravel(), bQ.ravel()])
    assert np.median(b / move) < 1e-2


@pytest.mark.parametrize("mistake", ["lambda", "drop", "sign", "factor"])
def test_planted_mistakes_fail_the_bound(case, mistake):
    bp, tr, P, Q = case
    Pn, Qn, _, bP, bQ, _ = _bound(case)
    P32, Q32, _ = _sweep32(bp, tr, P, Q, "forward", mistake=mistake)
    bad = np.sum(np.abs(P32 - Pn) > bP) + np.sum(np.abs(Q32 - Qn) > bQ)
    assert bad > 0


def test_bound_without_rounding_is_only_fp64(case):
    """u = 0 and u_store = 0: the bound shrinks to the FP64 slack, orders of
    magnitude below the FP32 bound at every entry."""
    bp, tr, P, Q = case
    args = (bp.U, bp.I, bp.user_offsets, bp.items, bp.ratings, *tr, P, Q, LAM, STEP)
    _, _, _, bP0, bQ0, bs0 = O.cf_sweep_bound(*args, u=0.0)
    _, _, _, bP, bQ, bs = O.cf_sweep_bound(*args)
    assert np.all(bP0 <= 1e-4 * bP) and np.all(bQ0 <= 1e-4 * bQ) and bs0 <= 1e-4 * bs


def test_selected_rows_equal_full_bound(case):
    """The bound at a selection of users and items equals the full bound at
    those rows (the selection only restricts the work)."""
    bp, tr, P, Q = case
    args = (bp.U, bp.I, bp.user_offsets, bp.items, bp.ratings, *tr, P, Q, LAM, STEP)
    _, _, _, bP, bQ, _ = O.cf_sweep_bound(*args)
    rng = np.random.default_rng(5)
    us = np.sort(rng.choice(bp.U, 50, replace=False))
    it = np.array([int(np.argmax(np.diff(tr[0]))), 0, bp.I - 1])
    _, _, _, sP, sQ, sb = O.cf_sweep_bound(*args, users=us, items=it)
    assert sb is None
    np.testing.assert_allclose(sP, bP[us], rtol=1e-12, atol=0)
    np.testing.assert_allclose(sQ, bQ[it], rtol=1e-12, atol=0)


def test_bf16_pair_storage_rounding_pinned():
    """The storage readings the bounds rely on: a BF16 value is x rounded to
    8 significant bits (relative error <= 2^-8), and a hi + lo pair is
    within 2^-16 |x| of x with hi + lo exact in FP32 (so decoding the pair
    adds no rounding)."""
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(200_000) * np.exp2(rng.integers(-30, 30, 200_000))).astype(np.float32)
    x = x[x != 0]
    h = _bf16(x).astype(np.float64)
    x64 = x.astype(np.float64)
    assert np.all(np.abs(h - x64) <= O.U_BF16 * np.abs(x64))
    hi = _bf16(x)
    lo = _bf16((x - hi).astype(np.float32))
    exact = hi.astype(np.float64) + lo.astype(np.float64)
    assert np.array_equal((hi + lo).astype(np.float64), exact)  # the FP32 sum is exact
    assert np.all(np.abs(exact - x64) <= O.U_BF16X2 * np.abs(x64))
