"""Thin Python binding of the cagra_gb C ABI (include/cagra_gb.h).

Argument marshalling only: torch tensors are passed as raw device pointers,
the current torch CUDA stream as the stream, and every status code is turned
into an exception.  All computation happens in the CUDA library; there is no
CPU fallback: if the library is missing or no GPU is present the calls fail.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcagra_gb.so")
_lock = threading.Lock()
_lib = None

CG_OP_SUM_F32 = 0
CG_OP_MIN_I32 = 1

# Every symbol include/cagra_gb.h declares (checked by the CPU test suite).
EXPORTS = [
    "cg_status_string", "cg_last_error_message", "cg_version",
    "cg_out_degree", "cg_inv_outdeg", "cg_cluster", "cg_relabel_csr", "cg_permute4",
    "cg_permute_rows",
    "pr_build_segments", "cg_segmented_get_info", "cg_segmented_stats", "pr_plan_bounds", "pr_set_gather_config",
    "pr_gather_table_capacity", "pr_set_gather_overlap", "cg_segmented_export",
    "cg_segmented_destroy", "cg_seg_gather", "cg_seg_gather_phases", "merge",
    "pr_init", "pr_contrib", "pr_iterate", "pr_merge_update", "pr_plain_create", "pr_plain_destroy", "pr_iterate_plain",
    "pr_iterate_plain_noalloc", "pr_noalloc_limits",
    "lp_iterate", "lp_run",
    "pr_batch_create", "pr_batch_destroy", "pr_batch_set_threads", "pr_batch_run",
    "pr_batched_graphs_run",
    "pr_init_ppr", "pr_iterate_ppr",
    "ppr_batched_create", "ppr_batched_destroy", "ppr_batched_bytes", "ppr_batched_init",
    "ppr_batched_iterate", "ppr_batched_step",
    "cf_transpose", "cf_create", "cf_destroy", "cf_set_factors", "cf_get_factors", "cf_sweep",
    "cf_sweep_phase", "cf_info",
    "cg_permute8", "cg_transpose_csr", "bc_create", "bc_destroy", "bc_set_direction", "bc_run",
    "bc_source_state", "cg_split_hub_block", "ppr_batched_attach_dense", "pr_set_gather_affine",
]


class CagraError(RuntimeError):
    pass


class SegInfo(ctypes.Structure):
    _fields_ = [("V", ctypes.c_int32), ("E", ctypes.c_int64), ("num_segments", ctypes.c_int32),
                ("merge_block", ctypes.c_int32), ("num_blocks", ctypes.c_int32),
                ("rows", ctypes.c_int64), ("q", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("gather_tiles", ctypes.c_int64),
                ("table_vertices", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("gather_threads", ctypes.c_int32), ("staged_segments", ctypes.c_int32),
                ("staged_edges", ctypes.c_int64), ("gather_overlap", ctypes.c_int32),
                ("affine_segments", ctypes.c_int32), ("affine_edges", ctypes.c_int64)]


def load(path: str | None = None):
    """Load libcagra_gb.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise CagraError(f"cagra_gb CUDA library not found at {p}; build it with "
                             "paper_1608_01362_gb300.build.build()")
        lib = ctypes.CDLL(p)
        i32, i64, dbl, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        sig = {
            "cg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "cg_last_error_message": (ctypes.c_char_p, []),
            "cg_version": (ctypes.c_int, []),
            "cg_out_degree": (ctypes.c_int, [vp, i64, i32, vp, vp]),
            "cg_inv_outdeg": (ctypes.c_int, [vp, i32, vp, vp]),
            "cg_cluster": (ctypes.c_int, [vp, i32, i64, i32, vp, vp, vp]),
            "cg_relabel_csr": (ctypes.c_int, [vp, vp, i32, i64, vp, vp, vp, vp, vp]),
            "cg_permute4": (ctypes.c_int, [vp, i64, vp, i64, vp, vp]),
            "cg_permute_rows": (ctypes.c_int, [vp, i64, i32, vp, i64, vp, vp]),
            "cg_permute8": (ctypes.c_int, [vp, i64, vp, i64, vp, vp]),
            "pr_build_segments": (ctypes.c_int, [vp, vp, i32, i64, i32, vp, i32,
                                                 ctypes.POINTER(vp), vp]),
            "cg_segmented_get_info": (ctypes.c_int, [vp, ctypes.POINTER(SegInfo)]),
            "cg_segmented_stats": (ctypes.c_int, [vp, vp, vp, vp]),
            "pr_plan_bounds": (ctypes.c_int, [vp, i32, i32, dbl, i32, i32, vp, vp, vp]),
            "pr_set_gather_config": (ctypes.c_int, [vp, i32, i32, i32, vp]),
            "pr_gather_table_capacity": (ctypes.c_int, [i32]),
            "pr_set_gather_overlap": (ctypes.c_int, [vp, i32, vp]),
            "pr_set_gather_affine": (ctypes.c_int, [vp, dbl, vp]),
            "cg_segmented_export": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, vp, vp]),
            "cg_segmented_destroy": (ctypes.c_int, [vp]),
            "cg_seg_gather": (ctypes.c_int, [vp, i32, vp, vp, vp]),
            "cg_seg_gather_phases": (ctypes.c_int, [vp, i32, vp, vp, i32, vp]),
            "merge": (ctypes.c_int, [vp, i32, vp, vp, vp]),
            "pr_init": (ctypes.c_int, [vp, i32, vp, vp, vp, vp]),
            "pr_contrib": (ctypes.c_int, [vp, vp, i32, vp, vp, vp]),
            "pr_iterate": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, dbl, i32, vp, vp, vp]),
            "pr_merge_update": (ctypes.c_int, [vp, vp, vp, vp, vp, dbl, vp, vp, vp, vp]),
            "pr_plain_create": (ctypes.c_int, [vp, vp, i32, i64, ctypes.POINTER(vp), vp]),
            "pr_plain_destroy": (ctypes.c_int, [vp]),
            "pr_iterate_plain": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, dbl, i32, vp, vp, i32,
                                                vp]),
            "pr_iterate_plain_noalloc": (ctypes.c_int, [vp, vp, i32, i64, vp, vp, vp, vp, vp, dbl,
                                                        vp, vp, vp]),
            "pr_noalloc_limits": (ctypes.c_int, [vp, vp, vp]),
            "lp_iterate": (ctypes.c_int, [vp, vp, vp, vp, vp, vp]),
            "lp_run": (ctypes.c_int, [vp, vp, i64, vp, vp, vp]),
            "pr_batch_create": (ctypes.c_int, [i32, vp, vp, vp, ctypes.POINTER(vp), vp]),
            "pr_batch_destroy": (ctypes.c_int, [vp]),
            "pr_batch_set_threads": (ctypes.c_int, [vp, i32]),
            "pr_batch_run": (ctypes.c_int, [vp, i32, dbl, vp, vp, vp]),
            "pr_batched_graphs_run": (ctypes.c_int, [vp, i32, dbl, vp, vp, vp]),
            "pr_init_ppr": (ctypes.c_int, [vp, i32, i32, vp, vp, vp, vp]),
            "pr_iterate_ppr": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, dbl, i32, i32, vp, vp,
                                              vp]),
            "ppr_batched_create": (ctypes.c_int, [vp, i32, ctypes.POINTER(vp), vp]),
            "ppr_batched_destroy": (ctypes.c_int, [vp]),
            "ppr_batched_bytes": (ctypes.c_int, [vp, vp, vp]),
            "ppr_batched_init": (ctypes.c_int, [vp, vp, vp, vp]),
            "ppr_batched_iterate": (ctypes.c_int, [vp, vp, dbl, i32, vp, vp, vp]),
            "ppr_batched_step": (ctypes.c_int, [vp, vp, dbl, i32, vp, vp, vp, vp]),
            "cf_transpose": (ctypes.c_int, [i64, i64, vp, vp, vp, vp, vp, vp, vp]),
            "cf_create": (ctypes.c_int, [i64, i64, i32, i32, vp, vp, vp, vp, vp, vp,
                                         ctypes.POINTER(vp), vp]),
            "cf_destroy": (ctypes.c_int, [vp]),
            "cf_set_factors": (ctypes.c_int, [vp, vp, vp, vp]),
            "cf_get_factors": (ctypes.c_int, [vp, vp, vp, vp]),
            "cf_sweep": (ctypes.c_int, [vp, i32, dbl, dbl, vp, vp]),
            "cf_sweep_phase": (ctypes.c_int, [vp, i32, dbl, dbl, vp, vp]),
            "cf_info": (ctypes.c_int, [vp, vp, vp, vp, vp]),
            "cg_transpose_csr": (ctypes.c_int, [vp, vp, i32, i64, vp, vp, vp]),
            "cg_split_hub_block": (ctypes.c_int, [vp, vp, i32, i64, i32, vp, vp, vp,
                                                  ctypes.POINTER(i64), vp]),
            "ppr_batched_attach_dense": (ctypes.c_int, [vp, i32, vp, vp]),
            "bc_create": (ctypes.c_int, [vp, vp, vp, vp, i32, i64, ctypes.POINTER(vp), vp]),
            "bc_destroy": (ctypes.c_int, [vp]),
            "bc_set_direction": (ctypes.c_int, [vp, dbl]),
            "bc_run": (ctypes.c_int, [vp, vp, i32, vp, vp]),
            "bc_source_state": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int, what: str):
    if status != 0:
        lib = load()
        msg = lib.cg_last_error_message().decode(errors="replace")
        name = lib.cg_status_string(status).decode()
        raise CagraError(f"{what}: {name}: {msg}")


def _ptr(t) -> int | None:
    """Device pointer of a torch tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise CagraError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise CagraError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dtype_check(t, dtype, name):
    if t.dtype != dtype:
        raise CagraError(f"{name} must be {dtype}, got {t.dtype}")


# ------------------------------------------------------------------ degrees

def cg_out_degree(src, V: int, outdeg, stream=None):
    import torch
    _dtype_check(src, torch.int32, "src"); _dtype_check(outdeg, torch.int32, "outdeg")
    _check(load().cg_out_degree(_ptr(src), src.numel(), V, _ptr(outdeg), _stream(stream)),
           "cg_out_degree")


def cg_inv_outdeg(outdeg, inv, stream=None):
    _check(load().cg_inv_outdeg(_ptr(outdeg), outdeg.numel(), _ptr(inv), _stream(stream)),
           "cg_inv_outdeg")


def cg_cluster(outdeg, E: int, mode: int, new_of_old, old_of_new, stream=None):
    _check(load().cg_cluster(_ptr(outdeg), outdeg.numel(), E, mode, _ptr(new_of_old),
                             _ptr(old_of_new), _stream(stream)), "cg_cluster")


def cg_relabel_csr(offsets, src, new_of_old, old_of_new, out_offsets, out_src, stream=None):
    V = offsets.numel() - 1
    _check(load().cg_relabel_csr(_ptr(offsets), _ptr(src), V, src.numel(), _ptr(new_of_old),
                                 _ptr(old_of_new), _ptr(out_offsets), _ptr(out_src),
                                 _stream(stream)), "cg_relabel_csr")


def cg_permute4(x, idx, out, stream=None):
    """out[i] = x[idx[i]] for 4-byte element tensors."""
    if x.element_size() != 4 or out.element_size() != 4:
        raise CagraError("cg_permute4 needs 4-byte elements")
    _check(load().cg_permute4(_ptr(x), x.numel(), _ptr(idx), idx.numel(), _ptr(out),
                              _stream(stream)), "cg_permute4")


def cg_permute8(x, idx, out, stream=None):
    """out[i] = x[idx[i]] for 8-byte elements."""
    if x.element_size() != 8 or out.element_size() != 8:
        raise CagraError("cg_permute8 needs 8-byte elements")
    _check(load().cg_permute8(_ptr(x), x.numel(), _ptr(idx), idx.numel(), _ptr(out),
                              _stream(stream)), "cg_permute8")


def cg_permute_rows(x, idx, out, stream=None):
    """Row i of out = row idx[i] of x (2-D tensors, rows a multiple of 16 bytes)."""
    if x.dim() != 2 or out.dim() != 2 or x.shape[1] != out.shape[1] or x.dtype != out.dtype:
        raise CagraError("cg_permute_rows needs 2-D tensors of equal row shape and dtype")
    _check(load().cg_permute_rows(_ptr(x), x.shape[0], x.shape[1] * x.element_size(), _ptr(idx),
                                  idx.numel(), _ptr(out), _stream(stream)), "cg_permute_rows")


# ------------------------------------------------------------------ segmenting

class Segmented:
    """Owner of a cg_segmented handle (destroyed with the object)."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            try:
                load().cg_segmented_destroy(self.handle)
            finally:
                self.handle = None

    @property
    def info(self) -> dict:
        inf = SegInfo()
        _check(load().cg_segmented_get_info(self.handle, ctypes.byref(inf)),
               "cg_segmented_get_info")
        return {f: getattr(inf, f) for f, _ in SegInfo._fields_}

    def stats(self) -> tuple[int, float, int]:
        """(subgraph rows, expansion factor q, device bytes held)."""
        rows, q, nbytes = ctypes.c_int64(), ctypes.c_double(), ctypes.c_size_t()
        _check(load().cg_segmented_stats(self.handle, ctypes.byref(rows), ctypes.byref(q),
                                         ctypes.byref(nbytes)), "cg_segmented_stats")
        return rows.value, q.value, nbytes.value


def pr_build_segments(offsets, src, num_segments: int, bounds=None, merge_block: int = 512,
                      stream=None) -> Segmented:
    import torch
    _dtype_check(offsets, torch.int64, "offsets"); _dtype_check(src, torch.int32, "src")
    V = offsets.numel() - 1
    hb = None
    if bounds is not None:
        b = np.ascontiguousarray(np.asarray(bounds, dtype=np.int64))
        if b.shape != (num_segments + 1,):
            raise CagraError("bounds must have num_segments + 1 entries")
        hb = b.ctypes.data
    h = ctypes.c_void_p()
    _check(load().pr_build_segments(_ptr(offsets), _ptr(src) if src.numel() else None, V,
                                    src.numel(), num_segments, hb, merge_block, ctypes.byref(h),
                                    _stream(stream)), "pr_build_segments")
    return Segmented(h.value)


def pr_plan_bounds(outdeg, smem_vertices: int = -1, min_avg_degree: float = 64.0,
                   max_global_vertices: int = -1, k_max: int = 1024, stream=None):
    """Segment bounds for this GPU (host int64 array of k+1 entries)."""
    out = np.empty(k_max + 1, dtype=np.int64)
    k = ctypes.c_int32()
    _check(load().pr_plan_bounds(_ptr(outdeg), outdeg.numel(), smem_vertices, min_avg_degree,
                                 max_global_vertices, k_max, out.ctypes.data, ctypes.byref(k),
                                 _stream(stream)), "pr_plan_bounds")
    return out[:k.value + 1].copy()


def pr_set_gather_config(seg: Segmented, threads: int = 1024, ctas_per_sm: int = 1,
                         table_vertices: int = -1, stream=None):
    _check(load().pr_set_gather_config(seg.handle, threads, ctas_per_sm, table_vertices,
                                       _stream(stream)), "pr_set_gather_config")


def pr_set_gather_overlap(seg: Segmented, cached_warps: int, stream=None):
    _check(load().pr_set_gather_overlap(seg.handle, cached_warps, _stream(stream)),
           "pr_set_gather_overlap")


def pr_set_gather_affine(seg: Segmented, head_min_avg_degree: float, stream=None):
    """> 0: the segment-affine plan with that head threshold; 0: off."""
    _check(load().pr_set_gather_affine(seg.handle, float(head_min_avg_degree), _stream(stream)),
           "pr_set_gather_affine")


def pr_gather_table_capacity(ctas_per_sm: int = 1) -> int:
    return int(load().pr_gather_table_capacity(ctas_per_sm))


def cg_segmented_export(seg: Segmented, stream=None) -> dict:
    """Canonical flat layout as numpy arrays (host copies)."""
    import torch
    inf = seg.info
    k, rows, E, nb = inf["num_segments"], inf["rows"], inf["E"], inf["num_blocks"]
    hb = np.empty(k + 1, np.int64); hr = np.empty(k + 1, np.int64); he = np.empty(k + 1, np.int64)
    dev = torch.device("cuda")
    rp = torch.empty(rows + 1, dtype=torch.int64, device=dev)
    col = torch.empty(max(E, 1), dtype=torch.int32, device=dev)
    idx = torch.empty(max(rows, 1), dtype=torch.int32, device=dev)
    blk = torch.empty(k * (nb + 1), dtype=torch.int32, device=dev)
    _check(load().cg_segmented_export(seg.handle, hb.ctypes.data, hr.ctypes.data, he.ctypes.data,
                                      _ptr(rp), _ptr(col), _ptr(idx), _ptr(blk), _stream(stream)),
           "cg_segmented_export")
    return {"bounds": hb, "row_base": hr, "edge_base": he, "row_ptr": rp.cpu().numpy(),
            "col": col.cpu().numpy()[:E], "idx_map": idx.cpu().numpy()[:rows],
            "block_start": blk.cpu().numpy()}


def cg_seg_gather(seg: Segmented, op: int, x, interm=None, stream=None):
    _check(load().cg_seg_gather(seg.handle, op, _ptr(x), _ptr(interm), _stream(stream)),
           "cg_seg_gather")


PHASE_STAGED, PHASE_CACHED, PHASE_FIXUP = 1, 2, 4


def cg_seg_gather_phases(seg: Segmented, op: int, x, interm=None, phases: int = 7, stream=None):
    _check(load().cg_seg_gather_phases(seg.handle, op, _ptr(x), _ptr(interm), phases,
                                       _stream(stream)), "cg_seg_gather_phases")


def merge(seg: Segmented, op: int, interm, out, stream=None):
    _check(load().merge(seg.handle, op, _ptr(interm), _ptr(out), _stream(stream)), "merge")


# ------------------------------------------------------------------ PageRank

def pr_init(inv, rank, contrib, dangling, stream=None):
    _check(load().pr_init(_ptr(inv), inv.numel(), _ptr(rank), _ptr(contrib), _ptr(dangling),
                          _stream(stream)), "pr_init")


def pr_contrib(inv, rank, contrib, dangling, stream=None):
    _check(load().pr_contrib(_ptr(inv), _ptr(rank), inv.numel(), _ptr(contrib), _ptr(dangling),
                             _stream(stream)), "pr_contrib")


def pr_iterate(seg: Segmented, inv, rank_in, contrib_in, rank_out, contrib_out, damping: float,
               iterations: int, dangling, resid=None, stream=None):
    _check(load().pr_iterate(seg.handle, _ptr(inv), _ptr(rank_in), _ptr(contrib_in),
                             _ptr(rank_out), _ptr(contrib_out), damping, iterations,
                             _ptr(dangling), _ptr(resid), _stream(stream)), "pr_iterate")


def pr_merge_update(seg: Segmented, inv, rank_in, rank_out, contrib_out, damping: float,
                    D_in, D_out, resid=None, stream=None):
    _check(load().pr_merge_update(seg.handle, _ptr(inv), _ptr(rank_in), _ptr(rank_out),
                                  _ptr(contrib_out), damping, _ptr(D_in), _ptr(D_out),
                                  _ptr(resid), _stream(stream)), "pr_merge_update")


class Plain:
    """Owner of a cg_plain handle; keeps the CSR tensors alive."""

    def __init__(self, handle: int, offsets, src):
        self.handle = handle
        self._keep = (offsets, src)

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            try:
                load().pr_plain_destroy(self.handle)
            finally:
                self.handle = None


def pr_plain_create(offsets, src, stream=None) -> Plain:
    import torch
    _dtype_check(offsets, torch.int64, "offsets"); _dtype_check(src, torch.int32, "src")
    h = ctypes.c_void_p()
    _check(load().pr_plain_create(_ptr(offsets), _ptr(src) if src.numel() else None,
                                  offsets.numel() - 1, src.numel(), ctypes.byref(h),
                                  _stream(stream)), "pr_plain_create")
    return Plain(h.value, offsets, src)


def pr_iterate_plain(plain: Plain, inv, rank_in, contrib_in, rank_out, contrib_out,
                     damping: float, iterations: int, dangling, resid=None, probe: bool = False,
                     stream=None):
    _check(load().pr_iterate_plain(plain.handle, _ptr(inv), _ptr(rank_in), _ptr(contrib_in),
                                   _ptr(rank_out), _ptr(contrib_out), damping, iterations,
                                   _ptr(dangling), _ptr(resid), int(probe), _stream(stream)),
           "pr_iterate_plain")


def pr_iterate_plain_noalloc(offsets, src, inv, rank_in, contrib_in, rank_out, contrib_out,
                             damping: float, dangling, resid=None, stream=None):
    """One plain PageRank iteration using only the library's fixed scratch."""
    _check(load().pr_iterate_plain_noalloc(_ptr(offsets), _ptr(src) if src.numel() else None,
                                           offsets.numel() - 1, src.numel(), _ptr(inv),
                                           _ptr(rank_in), _ptr(contrib_in), _ptr(rank_out),
                                           _ptr(contrib_out), damping, _ptr(dangling),
                                           _ptr(resid), _stream(stream)),
           "pr_iterate_plain_noalloc")


def pr_noalloc_limits():
    mv, me, sb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().pr_noalloc_limits(ctypes.byref(mv), ctypes.byref(me), ctypes.byref(sb)),
           "pr_noalloc_limits")
    return {"max_vertices": mv.value, "max_edges": me.value, "scratch_bytes": sb.value}


# ------------------------------------------------------------------ label propagation

def lp_iterate(seg: Segmented, labels_in, labels_out, dev_changed=None, sync: bool = True,
               stream=None):
    """One pass; returns the number of changed labels when sync is True."""
    h = ctypes.c_int64()
    _check(load().lp_iterate(seg.handle, _ptr(labels_in), _ptr(labels_out), _ptr(dev_changed),
                             ctypes.byref(h) if sync else None, _stream(stream)), "lp_iterate")
    return h.value if sync else None


def lp_run(seg: Segmented, labels, max_passes: int = 1 << 20, stream=None):
    """Passes until no label changes; returns (passes, changes per pass)."""
    cap = min(max_passes, 1 << 16)
    ch = np.zeros(cap, dtype=np.int64)
    p = ctypes.c_int64()
    _check(load().lp_run(seg.handle, _ptr(labels), cap, ctypes.byref(p), ch.ctypes.data,
                         _stream(stream)), "lp_run")
    return p.value, ch[:p.value].copy()


def pr_init_ppr(inv, seed: int, rank, contrib, dangling, stream=None):
    _check(load().pr_init_ppr(_ptr(inv), inv.numel(), seed, _ptr(rank), _ptr(contrib),
                              _ptr(dangling), _stream(stream)), "pr_init_ppr")


def pr_iterate_ppr(seg: Segmented, inv, rank_in, contrib_in, rank_out, contrib_out,
                   damping: float, iterations: int, seed: int, dangling, resid=None,
                   stream=None):
    _check(load().pr_iterate_ppr(seg.handle, _ptr(inv), _ptr(rank_in), _ptr(contrib_in),
                                 _ptr(rank_out), _ptr(contrib_out), damping, iterations, seed,
                                 _ptr(dangling), _ptr(resid), _stream(stream)), "pr_iterate_ppr")


# ------------------------------------------------------------------ batched personalised PR

PPR_COLUMNS = 64


class PprBatch:
    """Owner of a cg_ppr handle (keeps its segmented graph alive)."""

    def __init__(self, handle: int, seg: Segmented, planes: int):
        self.handle = handle
        self.seg = seg
        self.planes = planes

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            try:
                load().ppr_batched_destroy(self.handle)
            finally:
                self.handle = None

    @property
    def bytes(self) -> int:
        b, c = ctypes.c_int64(), ctypes.c_int64()
        _check(load().ppr_batched_bytes(self.handle, ctypes.byref(b), ctypes.byref(c)),
               "ppr_batched_bytes")
        return int(b.value)

    @property
    def chunks(self) -> int:
        b, c = ctypes.c_int64(), ctypes.c_int64()
        _check(load().ppr_batched_bytes(self.handle, ctypes.byref(b), ctypes.byref(c)),
               "ppr_batched_bytes")
        return int(c.value)


def ppr_batched_create(seg: Segmented, planes: int = 2, stream=None) -> PprBatch:
    h = ctypes.c_void_p()
    _check(load().ppr_batched_create(seg.handle, planes, ctypes.byref(h), _stream(stream)),
           "ppr_batched_create")
    return PprBatch(h.value, seg, planes)


def ppr_batched_init(ppr: PprBatch, inv, seeds, stream=None):
    sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32))
    if sd.shape != (PPR_COLUMNS,):
        raise CagraError(f"ppr_batched_init: need {PPR_COLUMNS} seeds, got shape {sd.shape}")
    _check(load().ppr_batched_init(ppr.handle, _ptr(inv), sd.ctypes.data, _stream(stream)),
           "ppr_batched_init")


def ppr_batched_iterate(ppr: PprBatch, inv, damping: float, iterations: int, rank_out=None,
                        resid=None, stream=None):
    _check(load().ppr_batched_iterate(ppr.handle, _ptr(inv), damping, iterations,
                                      _ptr(rank_out), _ptr(resid), _stream(stream)),
           "ppr_batched_iterate")


def ppr_batched_step(ppr: PprBatch, inv, damping: float, phases: int = 7, rank_old=None,
                     rank_out=None, resid=None, stream=None):
    _check(load().ppr_batched_step(ppr.handle, _ptr(inv), damping, phases, _ptr(rank_old),
                                   _ptr(rank_out), _ptr(resid), _stream(stream)),
           "ppr_batched_step")


# ------------------------------------------------------------------ collaborative filtering

CF_FP32, CF_BF16, CF_BF16X2 = 0, 1, 2


def cf_transpose(U: int, I: int, uoff, uitem, urate, ioff, iuser, irate, stream=None):
    _check(load().cf_transpose(U, I, _ptr(uoff), _ptr(uitem), _ptr(urate), _ptr(ioff),
                               _ptr(iuser), _ptr(irate), _stream(stream)), "cf_transpose")


class Bipartite:
    """Owner of a cg_bipartite handle (keeps the rating CSRs alive)."""

    def __init__(self, handle: int, keep):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            try:
                load().cf_destroy(self.handle)
            finally:
                self.handle = None

    @property
    def info(self) -> dict:
        v = [ctypes.c_int64() for _ in range(4)]
        _check(load().cf_info(self.handle, *[ctypes.byref(x) for x in v]), "cf_info")
        return dict(zip(("ratings", "user_pieces", "item_pieces", "bytes"),
                        [int(x.value) for x in v]))


def cf_create(U: int, I: int, K: int, precision: int, uoff, uitem, urate, ioff, iuser, irate,
              stream=None) -> Bipartite:
    h = ctypes.c_void_p()
    _check(load().cf_create(U, I, K, precision, _ptr(uoff), _ptr(uitem), _ptr(urate), _ptr(ioff),
                            _ptr(iuser), _ptr(irate), ctypes.byref(h), _stream(stream)),
           "cf_create")
    return Bipartite(h.value, (uoff, uitem, urate, ioff, iuser, irate))


def cf_set_factors(cf: Bipartite, P, Q, stream=None):
    _check(load().cf_set_factors(cf.handle, _ptr(P), _ptr(Q), _stream(stream)), "cf_set_factors")


def cf_get_factors(cf: Bipartite, P=None, Q=None, stream=None):
    _check(load().cf_get_factors(cf.handle, _ptr(P), _ptr(Q), _stream(stream)), "cf_get_factors")


def cf_sweep(cf: Bipartite, sweeps: int, lam: float, step: float, sse=None, stream=None):
    _check(load().cf_sweep(cf.handle, sweeps, lam, step, _ptr(sse), _stream(stream)), "cf_sweep")


def cf_sweep_phase(cf: Bipartite, phase: int, lam: float, step: float, sse=None, stream=None):
    _check(load().cf_sweep_phase(cf.handle, phase, lam, step, _ptr(sse), _stream(stream)),
           "cf_sweep_phase")


# ------------------------------------------------------------------ batched small graphs

class Batch:
    """Owner of a cg_batch handle."""

    def __init__(self, handle: int, G: int, vbase):
        self.handle = handle
        self.G = G
        self.vbase = vbase

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            try:
                load().pr_batch_destroy(self.handle)
            finally:
                self.handle = None


def pr_batch_create(vbase, offsets, src, stream=None) -> Batch:
    vb = np.ascontiguousarray(np.asarray(vbase, dtype=np.int64))
    G = vb.shape[0] - 1
    h = ctypes.c_void_p()
    _check(load().pr_batch_create(G, vb.ctypes.data, _ptr(offsets), _ptr(src), ctypes.byref(h),
                                  _stream(stream)), "pr_batch_create")
    return Batch(h.value, G, vb)


def pr_batch_set_threads(batch: Batch, threads: int):
    _check(load().pr_batch_set_threads(batch.handle, threads), "pr_batch_set_threads")


def pr_batch_run(batch: Batch, iterations: int, damping: float, rank, resid=None, stream=None):
    _check(load().pr_batch_run(batch.handle, iterations, damping, _ptr(rank), _ptr(resid),
                               _stream(stream)), "pr_batch_run")


def pr_batched_graphs_run(batch: Batch, iterations: int, damping: float, rank, resid=None,
                          stream=None):
    _check(load().pr_batched_graphs_run(batch.handle, iterations, damping, _ptr(rank),
                                        _ptr(resid), _stream(stream)), "pr_batched_graphs_run")


def cg_split_hub_block(offsets, src, h: int, out_offsets, out_src, bits, stream=None) -> int:
    """Hub block [0, h) x [0, h) of an in-edge CSR into a bitmap, the rest into
    (out_offsets, out_src); returns the rest's edge count."""
    V = offsets.numel() - 1
    er = ctypes.c_int64()
    _check(load().cg_split_hub_block(_ptr(offsets), _ptr(src) if src.numel() else None, V,
                                     src.numel(), int(h), _ptr(out_offsets),
                                     _ptr(out_src) if out_src.numel() else None, _ptr(bits),
                                     ctypes.byref(er), _stream(stream)), "cg_split_hub_block")
    return int(er.value)


def ppr_batched_attach_dense(ppr, h: int, bits, stream=None):
    _check(load().ppr_batched_attach_dense(ppr.handle, int(h), _ptr(bits), _stream(stream)),
           "ppr_batched_attach_dense")
    ppr._dense_bits = bits  # keep the bitmap alive with the handle


# ------------------------------------------------------------------ betweenness centrality

def cg_transpose_csr(offsets, src, out_offsets, out_dst, stream=None):
    """Out-edge CSR of an in-edge CSR (rows in ascending destination order)."""
    V = offsets.numel() - 1
    _dtype_check(offsets, torch_int64(), "offsets")
    _dtype_check(src, torch_int32(), "src")
    _check(load().cg_transpose_csr(_ptr(offsets), _ptr(src) if src.numel() else None, V,
                                   src.numel(), _ptr(out_offsets),
                                   _ptr(out_dst) if out_dst.numel() else None, _stream(stream)),
           "cg_transpose_csr")


class Betweenness:
    """Owns a cg_bc handle (and keeps its CSR tensors alive)."""

    def __init__(self, handle: int, keep):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            load().bc_destroy(self.handle)
            self.handle = None


def bc_create(in_offsets, in_src, out_offsets, out_dst, stream=None) -> Betweenness:
    V = in_offsets.numel() - 1
    h = ctypes.c_void_p()
    _check(load().bc_create(_ptr(in_offsets), _ptr(in_src) if in_src.numel() else None,
                            _ptr(out_offsets), _ptr(out_dst) if out_dst.numel() else None, V,
                            in_src.numel(), ctypes.byref(h), _stream(stream)), "bc_create")
    return Betweenness(h.value, (in_offsets, in_src, out_offsets, out_dst))


def bc_set_direction(bc: Betweenness, alpha: float):
    _check(load().bc_set_direction(bc.handle, float(alpha)), "bc_set_direction")


def bc_run(bc: Betweenness, sources, out, stream=None):
    """Adds the dependencies of every source (host IDs) into out (FP64[V])."""
    src = (ctypes.c_int32 * len(sources))(*[int(x) for x in sources])
    _dtype_check(out, torch_float64(), "out")
    _check(load().bc_run(bc.handle, src, len(sources), _ptr(out), _stream(stream)), "bc_run")


def bc_source_state(bc: Betweenness, level=None, sigma=None, delta=None, stream=None) -> dict:
    """The last source's level / sigma / delta into the given device tensors;
    returns {depth, push_levels, pull_levels}."""
    d, pu, pl = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().bc_source_state(bc.handle, _ptr(level), _ptr(sigma), _ptr(delta),
                                  ctypes.byref(d), ctypes.byref(pu), ctypes.byref(pl),
                                  _stream(stream)), "bc_source_state")
    return {"depth": d.value, "push_levels": pu.value, "pull_levels": pl.value}


def torch_int64():
    import torch
    return torch.int64


def torch_int32():
    import torch
    return torch.int32


def torch_float64():
    import torch
    return torch.float64


