"""Pins of the oracle's per-vertex rounding-error bound (oracle.pagerank_bound,
the PageRank iteration of Algorithms 1 and 5 and its personalised column).

The bound claims: whatever order a reduced-precision evaluation sums each
vertex's in-edges in, however it splits and merges them (Algorithms 3 and 4),
its result stays within bound[v] of the FP64 iterate at every vertex.  These
tests evaluate the iteration in FP32 (and with BF16 / BF16 hi+lo stored
contributions) in numpy, in several summation orders, and check the claim
element by element; they also check that the bound is not vacuous (an actual
evaluation comes within a small factor of it) and that it does fail a
planted mistake (one dropped edge).  CPU only."""
import numpy as np
import pytest

import graphgen
import oracle as O

D = O.DAMPING


def _bf16(x):
    """Round float32 values to BF16 (round to nearest, ties to even)."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _hilo(x):
    """Store as a BF16 pair hi = bf16(x), lo = bf16(x - hi); hi + lo is exact
    in FP32."""
    x = np.asarray(x, np.float32)
    h = _bf16(x)
    lo = _bf16((x - h).astype(np.float32))
    return (h + lo).astype(np.float32)


def _add_toward_zero(a, b):
    """FP32 a + b rounded toward zero, for non-negative a and b.  Their FP64
    sum is exact when the exponents differ by at most 29; otherwise the
    smaller operand lies below the FP32 result's last bit, FP64 rounds it
    by less than that, and truncation drops it either way."""
    y = a.astype(np.float64) + b.astype(np.float64)
    f = y.astype(np.float32)
    over = np.abs(f.astype(np.float64)) > np.abs(y)
    f[over] = np.nextafter(f[over], np.float32(0.0))
    return f


def _row_sums32(offsets, src, c, order, rng=None, drop=None):
    """Per-row FP32 sums of c[src[e]] in the given association order
    ("truncated": left to right, every addition rounded toward zero)."""
    V = len(offsets) - 1
    deg = np.diff(offsets)
    vals = c[src].astype(np.float32)
    if drop is not None:
        vals = vals.copy()
        vals[drop] = np.float32(0.0)
    if order == "truncated":
        acc = np.zeros(V, np.float32)
        for j in range(int(deg.max(initial=0))):
            m = deg > j
            acc[m] = _add_toward_zero(acc[m], vals[offsets[:-1][m] + j])
        return acc
    if order in ("forward", "reverse", "shuffled"):
        idx = np.arange(len(src))
        if order == "shuffled":
            idx = idx.copy()
            for v in range(V):
                lo, hi = offsets[v], offsets[v + 1]
                idx[lo:hi] = lo + rng.permutation(hi - lo)
        acc = np.zeros(V, np.float32)
        for j in range(int(deg.max(initial=0))):
            m = deg > j
            pos = offsets[:-1][m] + (j if order != "reverse" else deg[m] - 1 - j)
            acc[m] = (acc[m] + vals[idx[pos]]).astype(np.float32)
        return acc
    assert order == "pairwise"  # balanced tree over each row (zero padding is exact)
    w = 1
    while w < max(int(deg.max(initial=0)), 1):
        w *= 2
    A = np.zeros((V, w), np.float32)
    rows = np.repeat(np.arange(V), deg)
    A[rows, np.arange(len(src)) - offsets[:-1][rows]] = vals
    while A.shape[1] > 1:
        A = (A[:, 0::2] + A[:, 1::2]).astype(np.float32)
    return A[:, 0]


def _pagerank32(g, iters, seed=-1, order="forward", store=None, drop=None, rng_seed=0,
                base_fp32=False, dangling_parts=0):
    """The iteration evaluated in FP32 (FP64 dangling sum, as the GPU path).
    base_fp32: form (1-d)/V in FP32 from the rounded d (as the small-graph
    batch kernel does) instead of rounding the FP64 value once.
    dangling_parts > 0: the dangling mass from FP32 partial sums of that many
    consecutive dangling ranks, added in FP64 (as the GPU's update kernels)."""
    V = g.V
    rng = np.random.default_rng(rng_seed)
    outdeg = np.bincount(g.src, minlength=V)
    inv = np.zeros(V, np.float32)
    inv[outdeg > 0] = np.float32(1.0) / outdeg[outdeg > 0].astype(np.float32)
    d32 = np.float32(D)
    base32 = np.float32((1.0 - D) / V)
    if base_fp32:
        base32 = np.float32((np.float32(1.0) - d32) / np.float32(V))
    if seed < 0:
        r = np.full(V, np.float32(1.0) / np.float32(V), np.float32)
    else:
        r = np.zeros(V, np.float32)
        r[seed] = 1.0
    for _ in range(iters):
        Dm = float(np.sum(r[outdeg == 0].astype(np.float64)))
        if dangling_parts > 0:
            rd = r[outdeg == 0]
            Dm = 0.0
            for i in range(0, len(rd), dangling_parts):
                part = np.float32(0.0)
                for x in rd[i:i + dangling_parts]:
                    part = np.float32(part + x)
                Dm += float(part)
        c = (r * inv).astype(np.float32)
        if store is not None:
            c = store(c)
        s = _row_sums32(g.offsets, g.src, c, order, rng, drop)
        if seed < 0:
            Dv = np.float32(Dm * (1.0 / V))
            r = (base32 + (d32 * ((s + Dv).astype(np.float32))).astype(np.float32)).astype(
                np.float32)
        else:
            r = (d32 * s).astype(np.float32)
            r[seed] = np.float32(r[seed] + np.float32((1.0 - D) + D * Dm))
    return r


def _graphs():
    rng = np.random.default_rng(4)
    n = 3000
    return {
        "rmat10": graphgen.rmat(10, 16, seed=2),
        "in_star": graphgen.from_edges(n + 1, np.arange(1, n + 1), np.zeros(n, dtype=int)),
        "cycle": graphgen.from_edges(500, np.arange(500), (np.arange(500) + 1) % 500),
        "ragged": graphgen.from_edges(600, rng.integers(0, 600, 4000),
                                      (rng.integers(0, 600, 4000) ** 2) % 600),
    }


GRAPHS = _graphs()


def test_bound_rank_is_the_oracle_iterate():
    for g in GRAPHS.values():
        r, b = O.pagerank_bound(g.offsets, g.src, iters=20)
        want, _ = O.pagerank(g.offsets, g.src, iters=20)
        assert np.array_equal(r, want)
        assert np.all(b > 0)
        seeds = np.array([0, g.V // 2, g.V - 1], dtype=np.int32)
        R = O.ppr(g.offsets, g.src, seeds, iters=20)
        for j, s in enumerate(seeds):
            c, _ = O.pagerank_bound(g.offsets, g.src, iters=20, seed=int(s))
            assert np.array_equal(c, R[:, j])


def test_bound_without_rounding_is_only_fp64():
    g = GRAPHS["rmat10"]
    r, b = O.pagerank_bound(g.offsets, g.src, iters=20, u_acc=0.0, u_store=0.0)
    # what is left is this FP64 evaluation's own rounding, (n + 8 + 2V) 2^-53
    # per iteration (about 2e-13 here), accumulated over 20 iterations
    assert np.all(b <= 1e-11 * r)


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("order", ["forward", "reverse", "pairwise", "shuffled"])
def test_fp32_evaluations_stay_inside_the_bound(name, order):
    g = GRAPHS[name]
    want, bound = O.pagerank_bound(g.offsets, g.src, iters=20)
    for base_fp32 in (False, True):
        got = _pagerank32(g, 20, order=order, rng_seed=7, base_fp32=base_fp32)
        err = np.abs(got.astype(np.float64) - want)
        assert np.all(err <= bound), float(np.max(err / bound))


@pytest.mark.parametrize("name", ["rmat10", "ragged"])
def test_fp32_dangling_partials_stay_inside_the_bound(name):
    """The bound covers a dangling mass formed from FP32 partial sums of up
    to 256 ranks (the update kernels' per-lane partials) before FP64."""
    g = GRAPHS[name]
    want, bound = O.pagerank_bound(g.offsets, g.src, iters=20)
    for parts in (16, 256):
        got = _pagerank32(g, 20, order="forward", dangling_parts=parts)
        err = np.abs(got.astype(np.float64) - want)
        assert np.all(err <= bound), float(np.max(err / bound))


@pytest.mark.parametrize("store,u_store", [(_hilo, O.U_BF16X2), (_bf16, O.U_BF16),
                                           (None, 0.0)])
def test_personalised_column_with_stored_contributions_inside_the_bound(store, u_store):
    for g in (GRAPHS["rmat10"], GRAPHS["ragged"]):
        seed = int(np.argmax(np.bincount(g.src, minlength=g.V)))
        want, bound = O.pagerank_bound(g.offsets, g.src, iters=20, seed=seed, u_store=u_store)
        for order in ("forward", "pairwise"):
            got = _pagerank32(g, 20, seed=seed, order=order, store=store)
            assert np.all(np.abs(got.astype(np.float64) - want) <= bound)


@pytest.mark.parametrize("store,u_store", [(None, 0.0), (_hilo, O.U_BF16X2)])
def test_truncating_row_sums_inside_the_doubled_unit_bound(store, u_store):
    """The dense hub block's tensor-core sums may truncate instead of
    rounding to nearest; the parity tests of that path take the bound with
    u = 2^-23 (twice FP32's unit roundoff) for the row sums.  A personalised
    column whose every row-sum addition rounds toward zero stays inside that
    bound, and uses a visible share of it."""
    worst = 0.0
    for name in ("rmat10", "ragged", "cycle", "in_star"):
        g = GRAPHS[name]
        seed = int(np.argmax(np.bincount(g.src, minlength=g.V)))
        want, bound = O.pagerank_bound(g.offsets, g.src, iters=20, seed=seed,
                                       u_acc=2.0 ** -23, u_store=u_store)
        got = _pagerank32(g, 20, seed=seed, order="truncated", store=store)
        err = np.abs(got.astype(np.float64) - want)
        assert np.all(err <= bound), (name, float(np.max(err / bound)))
        m = bound > 0
        worst = max(worst, float(np.max(err[m] / bound[m])))
    assert worst >= 0.02


def test_toward_zero_addition_never_rounds_up():
    rng = np.random.default_rng(11)
    a = rng.random(100_000).astype(np.float32)
    b = (rng.random(100_000) * np.exp2(rng.integers(-30, 3, 100_000))).astype(np.float32)
    t = _add_toward_zero(a, b).astype(np.float64)
    exact = a.astype(np.float64) + b.astype(np.float64)
    n = (a + b).astype(np.float64)  # numpy: round to nearest
    assert np.all(t <= exact) and np.all(exact - t < np.spacing(t.astype(np.float32)))
    assert np.any(t < n)  # differs from round-to-nearest where nearest rounds up


def test_bound_is_not_vacuous():
    """Somewhere an actual FP32 evaluation comes within a factor of 100 of
    the bound (so the bound is a real constraint, not a blanket tolerance),
    and with BF16 storage within a factor of 10."""
    worst = 0.0
    for g in GRAPHS.values():
        want, bound = O.pagerank_bound(g.offsets, g.src, iters=20)
        for order in ("forward", "reverse"):
            got = _pagerank32(g, 20, order=order)
            worst = max(worst, float(np.max(np.abs(got - want) / bound)))
    assert worst >= 1e-2
    g = GRAPHS["rmat10"]
    seed = int(np.argmax(np.bincount(g.src, minlength=g.V)))
    want, bound = O.pagerank_bound(g.offsets, g.src, iters=20, seed=seed, u_store=O.U_BF16)
    got = _pagerank32(g, 20, seed=seed, store=_bf16)
    m = bound > 0  # vertices the seed cannot reach hold exactly 0 on both sides
    assert float(np.max(np.abs(got[m] - want[m]) / bound[m])) >= 0.1


@pytest.mark.parametrize("which", ["small_row", "hub_row"])
def test_bound_catches_one_dropped_edge(which):
    """A planted mistake (one in-edge left out of one row) breaks the bound."""
    g = GRAPHS["rmat10"]
    deg = np.diff(g.offsets)
    if which == "small_row":
        v = int(np.flatnonzero(deg == 3)[0])
    else:
        v = int(np.argmax(deg))
    want, bound = O.pagerank_bound(g.offsets, g.src, iters=20)
    got = _pagerank32(g, 20, drop=int(g.offsets[v]))
    assert np.any(np.abs(got.astype(np.float64) - want) > bound)
