"""ctypes declarations of the libh2gb C ABI (include/h2gb.h).

Argument marshalling only: every step of the construction runs in the CUDA
library.  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

# H2GB_LIB may point at another build of the library (e.g. a variant with
# different compile-time options).
LIB_PATH = os.environ.get("H2GB_LIB") or os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                      "libh2gb.so")

H2_OK = 0
H2_ERR_ARG = -1
H2_ERR_NOT_CONVERGED = -4
STATUS_NAMES = {0: "H2_OK", -1: "H2_ERR_ARG", -2: "H2_ERR_CUDA", -3: "H2_ERR_OOM",
                -4: "H2_ERR_NOT_CONVERGED", -5: "H2_ERR_TIMEOUT", -6: "H2_ERR_SAMPLER",
                -7: "H2_ERR_INPUT"}

SAMPLER_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                         C.c_int64, C.c_int, C.c_int64, C.c_void_p)


class BuildOpts(C.Structure):
    _fields_ = [("d0", C.c_int), ("d_inc", C.c_int), ("d_max", C.c_int), ("prec", C.c_int),
                ("omega_mode", C.c_int), ("seed", C.c_uint64),
                ("omega_stored", C.c_void_p), ("sketch", C.c_int), ("dense_a", C.c_void_p),
                ("sampler", SAMPLER_FN), ("sampler_ctx", C.c_void_p),
                ("operands", C.c_void_p), ("n_operands", C.c_int), ("timing", C.c_int),
                ("ksum_tile", C.c_int), ("lowrank_u", C.c_void_p), ("lowrank_v", C.c_void_p),
                ("lowrank_rank", C.c_int), ("bsr_engine", C.c_int), ("tc_cols", C.c_int),
                ("ksum_split", C.c_int), ("nonsym", C.c_int), ("psi_stored", C.c_void_p),
                ("sampler_t", SAMPLER_FN), ("sampler_t_ctx", C.c_void_p),
                ("queue_order", C.c_int), ("sum_engine", C.c_int)]


class TreeInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("dim", C.c_int), ("leaf_size", C.c_int), ("eta", C.c_double),
                ("depth", C.c_int), ("n_nodes", C.c_int), ("l_top", C.c_int),
                ("near_nnz", C.c_int64), ("far_nnz", C.c_int64 * 64)]


class Stats(C.Structure):
    _fields_ = [("count", C.c_int), ("n_total", C.c_int64), ("levels", C.c_int),
                ("d_final", C.c_int), ("rank_min", C.c_int), ("rank_max", C.c_int),
                ("converged", C.c_int), ("bytes_dense", C.c_int64),
                ("bytes_coupling", C.c_int64), ("bytes_basis", C.c_int64),
                ("near_entries", C.c_int64), ("sketch_pairs", C.c_int64),
                ("sketch_columns", C.c_int64), ("kernel_launches", C.c_int64),
                ("rounds", C.c_int), ("nrmK", C.c_double),
                ("ms_tree_unused", C.c_double), ("ms_sketch", C.c_double),
                ("ms_nearfield", C.c_double), ("ms_qr", C.c_double), ("ms_id", C.c_double),
                ("ms_upsweep", C.c_double), ("ms_coupling", C.c_double), ("ms_bsr", C.c_double),
                ("ms_total", C.c_double), ("ms_sketch_launch_max", C.c_double),
                ("sketch_flops", C.c_double), ("ms_sketch_kernel", C.c_double),
                ("sketch_launches", C.c_int64)]


vp = C.c_void_p
i64 = C.c_int64
i32 = C.c_int
dbl = C.c_double

# name -> (restype, argtypes); the same list the header declares
SIGNATURES = {
    "h2_default_opts": (None, [C.POINTER(BuildOpts)]),
    "h2_last_error": (C.c_char_p, []),
    "h2_kernel_launches": (C.c_int64, []),
    "h2_device_allocations": (C.c_int64, []),
    "h2_measure_peak": (C.c_int, [C.c_int, C.c_void_p, C.POINTER(C.c_double)]),
    "h2_trim_memory": (None, []),
    "h2_selftest_wait_timeout": (C.c_int, [C.c_void_p]),
    "h2_build_cluster_tree": (i32, [vp, i64, i32, i32, dbl, vp, C.POINTER(vp)]),
    "h2_tree_info": (i32, [vp, C.POINTER(TreeInfo)]),
    "h2_tree_export": (i32, [vp, vp, vp, vp, vp, vp]),
    "h2_tree_export_list": (i32, [vp, i32, i32, vp, vp]),
    "h2_tree_destroy": (None, [vp]),
    "h2_build": (i32, [vp, i32, vp, i32, dbl, C.POINTER(BuildOpts), vp, C.POINTER(vp)]),
    "h2_build_batched": (i32, [vp, i32, vp, vp, vp, C.POINTER(BuildOpts), vp, C.POINTER(vp)]),
    "h2_matvec": (i32, [vp, vp, vp, i32, vp]),
    "h2_stats": (i32, [vp, C.POINTER(Stats)]),
    "h2_export_level": (i32, [vp, i32, i32, vp, vp, vp, vp]),
    "h2_export_col_level": (i32, [vp, i32, i32, vp, vp]),
    "h2_matrix_destroy": (None, [vp]),
    "h2_autotune": (i32, [vp, i32, vp, i32, dbl, C.POINTER(BuildOpts), vp, C.POINTER(BuildOpts),
                          C.POINTER(dbl)]),
    "h2_ksum_sketch": (i32, [vp, i64, i32, i32, vp, i32, vp, i64, vp, i64, i32, i32, vp]),
    "h2_entry_block": (i32, [vp, i64, i32, i32, vp, i32, vp, i64, vp, i64, vp, vp]),
    "h2_dense_sketch": (i32, [vp, i64, i64, vp, i64, vp, i64, i32, vp]),
    "h2_batched_qr_mindiag": (i32, [i32, vp, vp, vp, vp, vp, vp]),
    "h2_batched_row_id": (i32, [i32, vp, vp, vp, vp, vp, vp, vp, i32, vp, vp, vp]),
    "h2_batched_qr_mindiag_static": (i32, [i32, vp, vp, vp, vp, vp, vp]),
}

_lib = None


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() or "
                               "python -m paper_2506_16759_gb300.build first")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class H2Error(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().h2_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str, allow=(H2_OK,)) -> int:
    if status not in allow:
        raise H2Error(status, where)
    return status
