"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module holds no arithmetic of the method itself (no PageRank, no
segmenting, no clustering): it draws SplitMix64 random numbers, generates
RMAT edges and Netflix-shaped bipartite ratings, drops self-loops and
duplicates, and lays the result out as an in-edge CSR (rows = destinations,
each row's sources ascending).  The C source is ``graphgen.c``; it is compiled
in-tree on first use (or by ``build()``).

Graph shapes follow the paper's workloads (Table I: RMAT graphs generated
with a/b/c/d = 0.57/0.19/0.19/0.05, self-loops and duplicates removed;
Netflix-shaped bipartite ratings).  Every generator is deterministic in its
seed and independent of the number of threads used.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "_graphgen.so")
_lock = threading.Lock()
_lib = None

RMAT_A, RMAT_B, RMAT_C = 0.57, 0.19, 0.19


def build(force: bool = False) -> str:
    """Compile graphgen.c into an in-tree shared library; returns its path."""
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
            i64, i32, u64, dbl, vp = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                      ctypes.c_double, ctypes.c_void_p)
            lib.gg_rmat_in_csr.restype = i64
            lib.gg_rmat_in_csr.argtypes = [i32, i32, dbl, dbl, dbl, u64, i32, i32, vp,
                                           ctypes.POINTER(vp)]
            lib.gg_edges_in_csr.restype = i64
            lib.gg_edges_in_csr.argtypes = [i64, i64, vp, vp, vp, ctypes.POINTER(vp)]
            lib.gg_bipartite.restype = i64
            lib.gg_bipartite.argtypes = [i64, i64, i64, dbl, dbl, dbl, u64, vp, vp, vp]
            lib.gg_permutation.restype = ctypes.c_int
            lib.gg_permutation.argtypes = [u64, i64, vp]
            lib.gg_splitmix_draws.restype = ctypes.c_int
            lib.gg_splitmix_draws.argtypes = [u64, u64, i32, vp]
            lib.gg_uniform_rows.restype = ctypes.c_int
            lib.gg_uniform_rows.argtypes = [u64, i64, i32, dbl, vp]
            lib.gg_free.restype = None
            lib.gg_free.argtypes = [vp]
            lib.gg_num_threads.restype = ctypes.c_int
            lib.gg_num_threads.argtypes = []
            _lib = lib
    return _lib


@dataclass
class CSR:
    """In-edge CSR: row v lists the sources of the edges u -> v."""
    offsets: np.ndarray  # int64[V+1]
    src: np.ndarray      # int32[E]

    @property
    def V(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def E(self) -> int:
        return int(self.offsets[-1])


def _take_src(lib, ptr: ctypes.c_void_p, E: int) -> np.ndarray:
    out = np.empty(E, dtype=np.int32)
    if E:
        ctypes.memmove(out.ctypes.data, ptr.value, E * 4)
    lib.gg_free(ptr)
    return out


def rmat(scale: int, edge_factor: int = 16, seed: int = 1, symmetric: bool = False,
         permute: bool = True, a: float = RMAT_A, b: float = RMAT_B,
         c: float = RMAT_C) -> CSR:
    """RMAT graph with 2**scale vertices as a cleaned in-edge CSR."""
    lib = _load()
    V = 1 << scale
    offsets = np.empty(V + 1, dtype=np.int64)
    ptr = ctypes.c_void_p()
    E = lib.gg_rmat_in_csr(scale, edge_factor, a, b, c, seed, int(symmetric), int(permute),
                           offsets.ctypes.data, ctypes.byref(ptr))
    if E < 0:
        raise MemoryError("graphgen: RMAT generation failed")
    return CSR(offsets, _take_src(lib, ptr, E))


def from_edges(V: int, src, dst) -> CSR:
    """Cleaned in-edge CSR (sorted rows, no self-loops, no duplicates)."""
    lib = _load()
    s = np.ascontiguousarray(np.asarray(src, dtype=np.int32))
    d = np.ascontiguousarray(np.asarray(dst, dtype=np.int32))
    if s.shape != d.shape:
        raise ValueError("src and dst differ in length")
    if s.size and (s.min() < 0 or d.min() < 0 or s.max() >= V or d.max() >= V):
        raise ValueError("edge endpoint out of range")
    offsets = np.empty(V + 1, dtype=np.int64)
    ptr = ctypes.c_void_p()
    E = lib.gg_edges_in_csr(V, s.size, s.ctypes.data, d.ctypes.data, offsets.ctypes.data,
                            ctypes.byref(ptr))
    if E < 0:
        raise MemoryError("graphgen: CSR build failed")
    return CSR(offsets, _take_src(lib, ptr, E))


def permutation(seed: int, n: int) -> np.ndarray:
    """Fisher-Yates permutation of 0..n-1 (perm[old] = new) from stream (seed, 0)."""
    out = np.empty(n, dtype=np.int32)
    _load().gg_permutation(seed, n, out.ctypes.data)
    return out


def splitmix_draws(seed: int, i: int, n: int) -> np.ndarray:
    """The first n uint64 draws of SplitMix64 stream (seed, i)."""
    out = np.empty(n, dtype=np.uint64)
    _load().gg_splitmix_draws(seed, i, n, out.ctypes.data)
    return out


def uniform_rows(seed: int, n: int, K: int, hi: float) -> np.ndarray:
    """n x K float64 matrix; row v holds the first K draws of SplitMix64
    stream (seed, v) mapped to [0, hi) (top 53 bits)."""
    out = np.empty((n, K), dtype=np.float64)
    if _load().gg_uniform_rows(seed, n, K, hi, out.ctypes.data) != 0:
        raise ValueError("graphgen: uniform_rows needs n >= 0 and K >= 1")
    return out


def cf_factors(U: int, I: int, K: int = 32, seed: int = 1):
    """Initial latent factors: entries uniform in [0, sqrt(12/K)) so that
    E[p . q] = 3 (the mean rating); users from seed, items from seed + 1."""
    hi = float(np.sqrt(12.0 / K))
    return uniform_rows(seed, U, K, hi), uniform_rows(seed + 1, I, K, hi)


@dataclass
class Bipartite:
    """User-major rating graph: user u rated items[user_offsets[u]:user_offsets[u+1]]."""
    U: int
    I: int
    user_offsets: np.ndarray  # int64[U+1]
    items: np.ndarray         # int32[R], ascending within each user
    ratings: np.ndarray       # uint8[R], values 1..5

    @property
    def R(self) -> int:
        return int(self.user_offsets[-1])


def bipartite(U: int = 480_189, I: int = 17_770, R: int = 99_000_000, mu: float = 4.4,
              sigma: float = 1.2, zipf_s: float = 1.0, seed: int = 1) -> Bipartite:
    """Netflix-shaped ratings: lognormal user degrees, Zipf item popularity."""
    lib = _load()
    offs = np.empty(U + 1, dtype=np.int64)
    items = np.empty(R, dtype=np.int32)
    ratings = np.empty(R, dtype=np.uint8)
    got = lib.gg_bipartite(U, I, R, mu, sigma, zipf_s, seed, offs.ctypes.data,
                           items.ctypes.data, ratings.ctypes.data)
    if got < 0:
        raise ValueError("graphgen: bipartite generation failed (bad sizes)")
    return Bipartite(U, I, offs, items[:got], ratings[:got])


def small_graph_batch(count: int = 1024, seed: int = 1, scale_lo: int = 8, scale_hi: int = 15,
                      edge_factor: int = 16):
    """`count` directed RMAT graphs.  Graph g takes two draws of SplitMix64
    stream (seed, g): the first gives its scale, uniform in [scale_lo,
    scale_hi] (the draw times the range count, high 64 bits), the second,
    cut to 63 bits, its RMAT seed.  Returns a list of CSR."""
    out = []
    for g in range(count):
        d = splitmix_draws(seed, g, 2)
        sc = scale_lo + int((int(d[0]) * (scale_hi - scale_lo + 1)) >> 64)
        out.append(rmat(sc, edge_factor, seed=int(d[1]) & 0x7FFFFFFFFFFFFFFF, permute=True))
    return out


def num_threads() -> int:
    return int(_load().gg_num_threads())
