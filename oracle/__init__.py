"""FP64 CPU oracle for the segmented pull gather of Cagra
("Making Caches Work for Graph Analytics", arXiv 1608.01362).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product path never does.
It is a plain, slow, obviously-correct restatement of what the hot path
computes, in FP64, sharing no code with the CUDA library (its C part is
``oracle.c``; the rest is numpy).  Each function cites the passage it follows.

Readings of the paper that the oracle fixes (the paper is silent or loose):
  * PageRank is the normalised form r_0 = 1/V,
    r'[v] = (1-d)/V + d (sum_{u->v} r[u]/outdeg(u) + D/V), D = rank mass of
    dangling vertices (Algorithm 5 prints the unnormalised 0.15 + 0.85 sum and
    divides by a possibly-zero out-degree); fixed iteration count, no early
    stop; d = 0.85.
  * Segments are contiguous source-ID ranges [bounds[s], bounds[s+1]); the
    paper's uniform choice is bounds[s] = min(s*N, V) with N = ceil(V/k)
    (Algorithm 2's segmentID = src / N).
  * Frequency-based clustering (Section V): mode 0 = stable sort by out-degree,
    descending (ties keep ascending vertex ID); mode 1 = stable sort by
    floor(outdeg / max(1, floor(E/V))), descending (the paper's "out-degree /
    threshold" with the average degree as threshold).
  * Label propagation is synchronous and includes the vertex's own label.
  * Collaborative filtering uses the degree-averaged gradient (see orc_cf_sweep).
  * Batched personalised PageRank returns dangling mass to each column's seed.

Pins (tests/test_oracle_pins.py): directed cycle, in-star closed form, rank
mass 1, dense brute-force power iteration and the linear-system fixed point,
Fig. 4's destination sets and expansion factor 7/6, segment invariants,
k = 1 segmented == plain bit for bit, label propagation == connected
components (scipy), reverse-path pass count, CF gradient == finite
differences of the loss, PPR column sums and one-hot equivalence.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

DAMPING = 0.85


def build(force: bool = False) -> str:
    """Compile oracle.c in-tree (gcc, OpenMP when available)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:2] + ["-fopenmp"] + base[2:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
            lib.orc_out_degree.restype = None
            lib.orc_out_degree.argtypes = [i64, vp, vp, vp]
            lib.orc_pagerank.restype = ctypes.c_int
            lib.orc_pagerank.argtypes = [i64, vp, vp, i32, dbl, vp, vp, vp]
            lib.orc_pagerank_bound.restype = ctypes.c_int
            lib.orc_pagerank_bound.argtypes = [i64, vp, vp, i32, dbl, i64, dbl, dbl, vp, vp, vp,
                                                vp]
            lib.orc_segments_count.restype = ctypes.c_int
            lib.orc_segments_count.argtypes = [i64, vp, vp, i32, vp, vp, vp]
            lib.orc_segments_fill.restype = ctypes.c_int
            lib.orc_segments_fill.argtypes = [i64, vp, vp, i32, vp, i64, vp, vp, vp, vp, vp, vp]
            lib.orc_pagerank_segmented.restype = ctypes.c_int
            lib.orc_pagerank_segmented.argtypes = [i64, i32, i64, vp, vp, vp, vp, vp, vp, i32,
                                                   dbl, vp, vp]
            lib.orc_label_propagation.restype = i64
            lib.orc_label_propagation.argtypes = [i64, vp, vp, vp, i64, vp]
            lib.orc_ppr.restype = ctypes.c_int
            lib.orc_ppr.argtypes = [i64, vp, vp, i32, vp, i32, dbl, vp]
            lib.orc_cf_sweep.restype = ctypes.c_int
            lib.orc_cf_sweep.argtypes = [i64, i64, i32, vp, vp, vp, vp, vp, vp, dbl, dbl, vp, vp,
                                         vp]
            lib.orc_out_csr.restype = ctypes.c_int
            lib.orc_out_csr.argtypes = [i64, vp, vp, vp, vp]
            lib.orc_bc_source.restype = i32
            lib.orc_bc_source.argtypes = [i64, vp, vp, i32, vp, vp, vp]
            lib.orc_num_threads.restype = ctypes.c_int
            lib.orc_num_threads.argtypes = []
            _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def num_threads() -> int:
    return int(_load().orc_num_threads())


# --------------------------------------------------------------------------
# Degrees (Algorithm 1's `degree` array; Algorithm 5's contrib = rank/outDegree)
# --------------------------------------------------------------------------

def out_degree(offsets, src) -> np.ndarray:
    """Out-degree of each vertex from an in-edge CSR (Section II-A)."""
    offsets = _c(offsets, np.int64)
    src = _c(src, np.int32)
    V = offsets.shape[0] - 1
    out = np.empty(V, dtype=np.int64)
    _load().orc_out_degree(V, offsets.ctypes.data, src.ctypes.data, out.ctypes.data)
    return out


# --------------------------------------------------------------------------
# PageRank (Algorithm 1 + Algorithm 5, normalised; see module docstring)
# --------------------------------------------------------------------------

def pagerank(offsets, src, iters: int = 20, d: float = DAMPING, rank0=None,
             iter_seconds=None):
    """Plain pull PageRank in FP64.  Returns (rank, residuals per iteration).
    iter_seconds: optional float64 array of length >= iters that receives the
    wall time of each iteration alone (set-up excluded)."""
    offsets = _c(offsets, np.int64)
    src = _c(src, np.int32)
    V = offsets.shape[0] - 1
    rank = np.full(V, 1.0 / V) if rank0 is None else _c(rank0, np.float64).copy()
    resid = np.zeros(max(iters, 1))
    secs = None
    if iter_seconds is not None:
        secs = iter_seconds
        assert secs.dtype == np.float64 and secs.flags.c_contiguous and secs.size >= iters
    if _load().orc_pagerank(V, offsets.ctypes.data, src.ctypes.data, iters, d, rank.ctypes.data,
                            resid.ctypes.data, 0 if secs is None else secs.ctypes.data) != 0:
        raise MemoryError("oracle: pagerank allocation failed")
    return rank, resid[:iters]


U_FP32 = 2.0 ** -24        # unit roundoff of FP32 arithmetic
U_BF16X2 = 2.0 ** -16      # relative rounding of a value stored as a BF16 hi + lo pair
U_BF16 = 2.0 ** -8         # relative rounding of a value stored as BF16


def pagerank_bound(offsets, src, iters: int = 20, d: float = DAMPING, seed: int = -1,
                   u_acc: float = U_FP32, u_store: float = 0.0, resid=None,
                   iter_seconds=None):
    """The PageRank iteration in FP64 (seed < 0: r_0 = 1/V, uniform teleport;
    seed >= 0: one personalised column, r_0 = one-hot) together with a
    per-vertex bound on the rounding error of any evaluation of it in a
    format of unit roundoff u_acc whose stored contributions carry a further
    relative rounding u_store (see orc_pagerank_bound for the recurrence).
    Returns (rank, bound): |r_computed - rank| <= bound element by element.
    rank equals pagerank(...)[0] (uniform) or ppr(...)[:, j] (personalised)
    bit for bit.  resid: optional float64 array (>= iters) that receives the
    per-iteration L1 residuals; iter_seconds as in pagerank (the bound's work
    excluded)."""
    offsets = _c(offsets, np.int64)
    src = _c(src, np.int32)
    V = offsets.shape[0] - 1
    rank = np.empty(V)
    bound = np.empty(V)
    secs = None
    if iter_seconds is not None:
        secs = iter_seconds
        assert secs.dtype == np.float64 and secs.flags.c_contiguous and secs.size >= iters
    if resid is not None:
        assert resid.dtype == np.float64 and resid.flags.c_contiguous and resid.size >= iters
    st = _load().orc_pagerank_bound(V, offsets.ctypes.data, src.ctypes.data, iters, d, int(seed),
                                    float(u_acc), float(u_store), rank.ctypes.data,
                                    bound.ctypes.data, 0 if resid is None else resid.ctypes.data,
                                    0 if secs is None else secs.ctypes.data)
    if st == -2:
        raise ValueError("oracle: pagerank_bound needs V >= 1 and seed < V")
    if st != 0:
        raise MemoryError("oracle: pagerank_bound allocation failed")
    return rank, bound


# --------------------------------------------------------------------------
# Frequency-based clustering (Section V)
# --------------------------------------------------------------------------

def cluster(outdeg, mode: int = 0, E: int | None = None):
    """Stable degree-driven renumbering.  Returns (new_of_old, old_of_new).

    mode 0: key = out-degree; mode 1: key = floor(outdeg / max(1, floor(E/V))).
    Vertices are ordered by key descending; equal keys keep their old order
    (the paper's parallel stable sort on out-degree/threshold)."""
    outdeg = np.asarray(outdeg, dtype=np.int64)
    V = outdeg.shape[0]
    if mode == 0:
        key = outdeg
    elif mode == 1:
        if E is None:
            E = int(outdeg.sum())
        thr = max(1, E // max(V, 1))
        key = outdeg // thr
    else:
        raise ValueError("mode must be 0 or 1")
    old_of_new = np.argsort(-key, kind="stable").astype(np.int32)
    new_of_old = np.empty(V, dtype=np.int32)
    new_of_old[old_of_new] = np.arange(V, dtype=np.int32)
    return new_of_old, old_of_new


def relabel(offsets, src, new_of_old, old_of_new):
    """Apply the renumbering to an in-edge CSR: new row n is old row
    old_of_new[n], each source replaced by new_of_old[source], in-row order
    kept (Section V: the mapping updates the vertex index in G.edgeArray)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    src = np.asarray(src, dtype=np.int32)
    old_of_new = np.asarray(old_of_new, dtype=np.int64)
    lens = np.diff(offsets)[old_of_new]
    noff = np.zeros(offsets.shape[0], dtype=np.int64)
    np.cumsum(lens, out=noff[1:])
    starts = offsets[old_of_new]
    # gather index of every new edge position
    pos = np.repeat(starts - noff[:-1], lens) + np.arange(noff[-1], dtype=np.int64)
    nsrc = np.asarray(new_of_old, dtype=np.int32)[src[pos]]
    return noff, nsrc.astype(np.int32)


# --------------------------------------------------------------------------
# Segmenting (Algorithm 2) and segmented PageRank (Algorithms 3, 4)
# --------------------------------------------------------------------------

def uniform_bounds(V: int, k: int) -> np.ndarray:
    """Algorithm 2's segments: N = ceil(V/k) vertices each, the last short."""
    N = -(-V // k) if V else 0
    return np.array([min(s * N, V) for s in range(k + 1)], dtype=np.int64)


@dataclass
class Segments:
    V: int
    k: int
    B: int
    bounds: np.ndarray       # int64[k+1]  source range of each segment
    row_base: np.ndarray     # int64[k+1]
    edge_base: np.ndarray    # int64[k+1]
    row_ptr: np.ndarray      # int64[rows+1]
    col: np.ndarray          # int32[E]
    idx_map: np.ndarray      # int32[rows]
    block_start: np.ndarray  # int32[k*(nb+1)]

    @property
    def rows(self) -> int:
        return int(self.row_base[-1])

    @property
    def nblocks(self) -> int:
        return -(-self.V // self.B)

    @property
    def q(self) -> float:
        """Expansion factor q = s_adj / s (Section III-D): the mean number of
        segments that contribute to a vertex = total subgraph rows / V."""
        return self.rows / self.V if self.V else 0.0


def build_segments(offsets, src, k: int | None = None, B: int = 2048, bounds=None) -> Segments:
    """Algorithm 2 (Section III-A): subgraphs of the in-edges grouped by source
    segment, each with idxMap, block indices for the merge and a CSR."""
    offsets = _c(offsets, np.int64)
    src = _c(src, np.int32)
    V = offsets.shape[0] - 1
    if bounds is None:
        bounds = uniform_bounds(V, k)
    bounds = _c(bounds, np.int64)
    k = bounds.shape[0] - 1
    if k < 1 or bounds[0] != 0 or bounds[-1] != V or np.any(np.diff(bounds) < 0) or B < 1:
        raise ValueError("bad segment bounds or block size")
    lib = _load()
    row_base = np.empty(k + 1, dtype=np.int64)
    edge_base = np.empty(k + 1, dtype=np.int64)
    if lib.orc_segments_count(V, offsets.ctypes.data, src.ctypes.data, k, bounds.ctypes.data,
                              row_base.ctypes.data, edge_base.ctypes.data) != 0:
        raise MemoryError("oracle: segment count failed")
    rows = int(row_base[-1])
    E = int(edge_base[-1])
    nb = -(-V // B)
    row_ptr = np.empty(rows + 1, dtype=np.int64)
    col = np.empty(max(E, 1), dtype=np.int32)
    idx_map = np.empty(max(rows, 1), dtype=np.int32)
    block_start = np.empty(k * (nb + 1), dtype=np.int32)
    if lib.orc_segments_fill(V, offsets.ctypes.data, src.ctypes.data, k, bounds.ctypes.data, B,
                             row_base.ctypes.data, edge_base.ctypes.data, row_ptr.ctypes.data,
                             col.ctypes.data, idx_map.ctypes.data,
                             block_start.ctypes.data) != 0:
        raise MemoryError("oracle: segment fill failed")
    return Segments(V, k, B, bounds, row_base, edge_base, row_ptr, col[:E], idx_map[:rows],
                    block_start)


def pagerank_segmented(seg: Segments, outdeg, iters: int = 20, d: float = DAMPING, rank0=None):
    """PageRank computed through the segmented structure, FP64 (Algorithms
    3 and 4 followed by the vertex update).  Returns (rank, residuals)."""
    V = seg.V
    outdeg = _c(outdeg, np.int64)
    rank = np.full(V, 1.0 / V) if rank0 is None else _c(rank0, np.float64).copy()
    resid = np.zeros(max(iters, 1))
    col = seg.col if seg.col.size else np.zeros(1, np.int32)
    idx = seg.idx_map if seg.idx_map.size else np.zeros(1, np.int32)
    if _load().orc_pagerank_segmented(V, seg.k, seg.B, seg.row_base.ctypes.data,
                                      seg.row_ptr.ctypes.data, col.ctypes.data, idx.ctypes.data,
                                      seg.block_start.ctypes.data, outdeg.ctypes.data, iters, d,
                                      rank.ctypes.data, resid.ctypes.data) != 0:
        raise MemoryError("oracle: segmented pagerank allocation failed")
    return rank, resid[:iters]


# --------------------------------------------------------------------------
# Label propagation (Table IV; min-label connected components)
# --------------------------------------------------------------------------

def label_propagation(offsets, src, labels0, max_passes: int = 1 << 30):
    """Synchronous min-label passes until no label changes.
    Returns (labels, passes, changes_per_pass)."""
    offsets = _c(offsets, np.int64)
    src = _c(src, np.int32)
    V = offsets.shape[0] - 1
    labels = _c(labels0, np.int32).copy()
    cap = min(max_passes, V + 2)
    changes = np.zeros(max(cap, 1), dtype=np.int64)
    p = _load().orc_label_propagation(V, offsets.ctypes.data, src.ctypes.data, labels.ctypes.data,
                                      cap, changes.ctypes.data)
    if p < 0:
        raise MemoryError("oracle: label propagation allocation failed")
    return labels, int(p), changes[:p]


def label_propagation_pass(offsets, src, labels):
    """Exactly one synchronous pass; returns (new_labels, changed)."""
    out, p, ch = label_propagation(offsets, src, labels, max_passes=1)
    return out, int(ch[0]) if p else 0


# --------------------------------------------------------------------------
# Batched personalised PageRank (64 columns)
# --------------------------------------------------------------------------

def ppr(offsets, src, seeds, iters: int = 20, d: float = DAMPING) -> np.ndarray:
    """Personalised PageRank for every seed at once; returns R[V, J] (FP64)."""
    offsets = _c(offsets, np.int64)
    src = _c(src, np.int32)
    seeds = _c(seeds, np.int32)
    V = offsets.shape[0] - 1
    J = seeds.shape[0]
    R = np.empty((V, J), dtype=np.float64)
    if _load().orc_ppr(V, offsets.ctypes.data, src.ctypes.data, J, seeds.ctypes.data, iters, d,
                       R.ctypes.data) != 0:
        raise MemoryError("oracle: ppr allocation failed")
    return R


# --------------------------------------------------------------------------
# Collaborative filtering (Table III)
# --------------------------------------------------------------------------

def item_major(U: int, I: int, user_offsets, items, ratings):
    """Transpose a user-major rating CSR into item-major (users ascending)."""
    user_offsets = np.asarray(user_offsets, dtype=np.int64)
    items = np.asarray(items, dtype=np.int64)
    users = np.repeat(np.arange(U, dtype=np.int64), np.diff(user_offsets))
    order = np.lexsort((users, items))
    ioff = np.zeros(I + 1, dtype=np.int64)
    np.cumsum(np.bincount(items, minlength=I), out=ioff[1:])
    return ioff, users[order].astype(np.int32), np.asarray(ratings, dtype=np.uint8)[order]


def cf_sweep(U, I, uoff, uitem, urate, ioff, iuser, irate, P, Q, lam=0.05, step=1e-3):
    """One Jacobi gradient sweep in FP64 (degree-averaged gradient).
    Returns (P', Q', sse of the old P, Q)."""
    P = _c(P, np.float64).copy()
    Q = _c(Q, np.float64).copy()
    K = P.shape[1]
    uoff, ioff = _c(uoff, np.int64), _c(ioff, np.int64)
    uitem, iuser = _c(uitem, np.int32), _c(iuser, np.int32)
    urate, irate = _c(urate, np.uint8), _c(irate, np.uint8)
    sse = ctypes.c_double()
    if _load().orc_cf_sweep(U, I, K, uoff.ctypes.data, uitem.ctypes.data, urate.ctypes.data,
                            ioff.ctypes.data, iuser.ctypes.data, irate.ctypes.data, lam, step,
                            P.ctypes.data, Q.ctypes.data, ctypes.byref(sse)) != 0:
        raise ValueError("oracle: cf sweep failed (K out of range or allocation)")
    return P, Q, float(sse.value)


def _gam(n, u=U_FP32):
    n = np.asarray(n, dtype=np.float64)
    return n * u / (1.0 - n * u)


def _side_bound(off, nbr, val, X, Y, Xn, lam, step, u, u_store, sel=None):
    """Per-entry bound of one side of a CF sweep (own factors X, neighbour
    factors Y, FP64 result Xn) at the vertices `sel` (None: all); see
    cf_sweep_bound.  Also returns per vertex the FP64 sum of e^2 and its error
    bound's two sums."""
    off = np.asarray(off, np.int64)
    if sel is not None:  # the selected vertices' rating lists as one CSR
        sel = np.asarray(sel, np.int64)
        sdeg = off[sel + 1] - off[sel]
        soff = np.zeros(len(sel) + 1, np.int64)
        np.cumsum(sdeg, out=soff[1:])
        idx = np.repeat(off[sel] - soff[:-1], sdeg) + np.arange(soff[-1])
        off, nbr, val = soff, np.asarray(nbr)[idx], np.asarray(val)[idx]
        X, Xn = X[sel], Xn[sel]
    n, K = X.shape
    deg = np.diff(off)
    rows = np.repeat(np.arange(n), deg)
    Yr = Y[np.asarray(nbr, np.int64)]
    prod = X[rows] * Yr
    S = np.abs(prod).sum(axis=1)
    e = np.asarray(val, np.float64) - prod.sum(axis=1)
    gK = _gam(K, u)
    de = gK * S + u * (np.abs(e) + gK * S)  # |fl(e) - e|: K-term dot, then r - dot

    def per_vertex(a):
        out = np.zeros((n,) + a.shape[1:])
        nz = deg > 0
        if nz.any():
            out[nz] = np.add.reduceat(a, off[:-1][nz], axis=0)
        return out

    absY = np.abs(Yr)
    G = per_vertex(e[:, None] * Yr)
    A1 = per_vertex(de[:, None] * absY)
    A2 = per_vertex((np.abs(e) + de)[:, None] * absY) * (1.0 + 1e-12)
    g2 = _gam(2, u)
    dg = np.maximum(deg, 1).astype(np.float64)[:, None]
    Eg = A1 + _gam(deg, u)[:, None] * A2           # any tree over deg products
    Ea = (Eg / dg) * (1.0 + g2) + g2 * np.abs(G) / dg  # times a rounded 1/deg
    Eb = g2 * lam * np.abs(X)                       # rounded lambda, one product
    c = G / dg - lam * X
    Ec = Ea + Eb + u * (np.abs(c) + Ea + Eb)
    Ed = step * ((1.0 + g2) * Ec + g2 * np.abs(c))  # rounded step, one product
    Ex = Ed + u * (np.abs(Xn) + Ed)                 # x + d
    slack = 2.0 ** -44 * (np.abs(X) + step * (np.abs(c) + A2 / dg + lam * np.abs(X)))
    bound = Ex + u_store * (np.abs(Xn) + Ex) + slack
    sse_v = per_vertex(e * e)
    sse_err_v = per_vertex(2.0 * np.abs(e) * de + de * de)
    return bound, deg, sse_v, sse_err_v


def cf_sweep_bound(U, I, uoff, uitem, urate, ioff, iuser, irate, P, Q, lam=0.05, step=1e-3,
                   u_store=0.0, piece=None, u=U_FP32, users=None, items=None):
    """One FP64 sweep (cf_sweep) and, per entry of P' and Q', a bound on how
    far a reduced-precision evaluation of the same sweep from the same P, Q
    can land from it; and a bound on its sum of squared errors.

    The evaluation it covers computes in arithmetic of unit roundoff u (FP32
    by default): each rating's dot product p_u . q_i with any summation tree
    (fused or separate multiply-adds), e = r - dot with one rounding, each
    vertex's gradient sum of e * y over its ratings with any summation tree,
    the division by deg as a rounded reciprocal and a product, lambda and the
    step rounded to that arithmetic, and x + step (g/deg - lambda x) with one
    rounding per operation; then it stores x' in a format of relative
    rounding u_store (0: FP32; U_BF16: BF16; U_BF16X2: a BF16 hi + lo pair).
    Standard bounds (Higham, Accuracy and Stability of Numerical Algorithms,
    Lemma 3.1 and Sec. 3.1): a sum of n terms in any tree has error at most
    gamma_{n-1} times the sum of the absolute terms, gamma_n = n u / (1 - n u).
    Per rating (S = sum_j |p_uj q_ij|):
        |fl(e) - e| <= gamma_K S + u (|e| + gamma_K S) =: de
    per vertex v and dimension k (the terms are e y_k; G = sum e y_k):
        |fl(G) - G| <= sum de |y_k| + gamma_deg sum (|e| + de) |y_k|
    and through the update, each rounding adding u times the magnitude of its
    result plus the error carried in.  The SSE is formed in partial sums of at
    most `piece` ratings of one user (None: all of them) in that arithmetic,
    combined in FP64.  Returns (P', Q', sse, bound_P, bound_Q, bound_sse);
    with `users` (`items`) given, bound_P (bound_Q) holds only those rows, in
    that order, and bound_sse is None unless every user is covered."""
    P64 = _c(P, np.float64)
    Q64 = _c(Q, np.float64)
    Pn, Qn, sse = cf_sweep(U, I, uoff, uitem, urate, ioff, iuser, irate, P64, Q64, lam, step)
    bP, udeg, sse_u, sse_err_u = _side_bound(uoff, uitem, urate, P64, Q64, Pn, lam, step, u,
                                             u_store, users)
    bQ = _side_bound(ioff, iuser, irate, Q64, P64, Qn, lam, step, u, u_store, items)[0]
    if users is not None:
        return Pn, Qn, sse, bP, bQ, None
    m = udeg if piece is None else np.minimum(udeg, piece)
    gm = _gam(m, u)
    b_sse = float(np.sum(sse_err_u * (1.0 + gm) + gm * sse_u))
    # FP64 combination of the partials, and the FP64 sum above
    b_sse += _gam(int(np.sum(udeg)) + len(udeg) + 4096, 2.0 ** -53) * float(np.sum(sse_u) + b_sse)
    return Pn, Qn, sse, bP, bQ, b_sse



# --------------------------------------------------------------------------
# Betweenness centrality (Table V: 12 sources; Brandes' algorithm)
# --------------------------------------------------------------------------

def out_csr(offsets, src):
    """Out-edge CSR (out_off, out_dst) of an in-edge CSR: row u lists the
    destinations of u's out-edges in ascending order (a counting sort)."""
    offsets = _c(offsets, np.int64)
    src = _c(src, np.int32)
    V = offsets.shape[0] - 1
    out_off = np.empty(V + 1, dtype=np.int64)
    out_dst = np.empty(max(src.shape[0], 1), dtype=np.int32)
    if _load().orc_out_csr(V, offsets.ctypes.data,
                           (src if src.size else np.zeros(1, np.int32)).ctypes.data,
                           out_off.ctypes.data, out_dst.ctypes.data) != 0:
        raise MemoryError("oracle: out_csr allocation failed")
    return out_off, out_dst[:src.shape[0]]


def bc_source(out_off, out_dst, s: int):
    """(level, sigma, delta, levels) of one source over an out-edge CSR."""
    out_off = _c(out_off, np.int64)
    out_dst = _c(out_dst, np.int32)
    V = out_off.shape[0] - 1
    level = np.empty(V, dtype=np.int32)
    sigma = np.empty(V)
    delta = np.empty(V)
    depth = _load().orc_bc_source(V, out_off.ctypes.data,
                                  (out_dst if out_dst.size else np.zeros(1, np.int32)).ctypes.data,
                                  int(s), level.ctypes.data, sigma.ctypes.data, delta.ctypes.data)
    if depth < 0:
        raise ValueError("oracle: bc source out of range or allocation failed")
    return level, sigma, delta, int(depth)


def betweenness(offsets, src, sources):
    """Betweenness centrality of every vertex from the given sources (sum over
    the sources s of the dependencies delta_s(v), v != s), FP64, on the graph
    given as an in-edge CSR.  Returns (bc, per-source (level, sigma, delta))."""
    out_off, out_dst = out_csr(offsets, src)
    V = out_off.shape[0] - 1
    bc = np.zeros(V)
    per = []
    for s in sources:
        level, sigma, delta, _ = bc_source(out_off, out_dst, int(s))
        d = delta.copy()
        d[int(s)] = 0.0
        bc += d
        per.append((level, sigma, delta))
    return bc, per
