"""ctypes declarations of the C ABI in include/gbspmv.h (marshalling only).

The shared library is loaded from this package directory.  A missing or
stale library raises immediately: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbspmv.so")

c_i32 = ctypes.c_int32
c_i64 = ctypes.c_int64
c_vp = ctypes.c_void_p
c_f32 = ctypes.c_float

# enums (values fixed by the header)
GBSP_OK = 0
STATUS = {0: "GBSP_OK", -1: "GBSP_ERR_ARG", -2: "GBSP_ERR_MATRIX", -3: "GBSP_ERR_CUDA",
          -4: "GBSP_ERR_NOMEM", -5: "GBSP_ERR_UNSUPPORTED", -6: "GBSP_ERR_TIMEOUT"}
F64, F32 = 0, 1
FORMATS = {"CRS": 0, "JDS": 1, "NBJDS": 2, "RBJDS": 3, "NUJDS": 4, "SOJDS": 5, "JDS_LITERAL": 6,
           "SELL": 7, "PSELL": 8}
PERM = {"symmetric": 0, "row_only": 1}
OP_N, OP_T = 0, 1
BASIS_PERMUTED, BASIS_ORIGINAL = 0, 1
ACC_PLAIN, ACC_COMPENSATED = 0, 1
KERNELS = {"auto": 0, "vector": 1, "tiled": 2, "runs": 3}


class KernelOpts(ctypes.Structure):
    _fields_ = [("kernel", c_i32), ("lanes", c_i32), ("rows_per_warp", c_i32), ("tile", c_i32),
                ("rhs_tile", c_i32), ("accum", c_i32), ("format", c_i32), ("block", c_i32),
                ("unroll", c_i32)]


class JdsOpts(ctypes.Structure):
    _fields_ = [("format", c_i32), ("perm_mode", c_i32), ("block", c_i32), ("unroll", c_i32),
                ("window", c_i32)]


class JdsSizes(ctypes.Structure):
    _fields_ = [("n_rows", c_i64), ("n_cols", c_i64), ("nnz", c_i64), ("n_diag", c_i64),
                ("n_blocks", c_i64), ("workspace_bytes", c_i64)]


class JdsBuffers(ctypes.Structure):
    _fields_ = [("jd_ptr", c_vp), ("col", c_vp), ("val", c_vp), ("perm", c_vp), ("iperm", c_vp),
                ("blk_ptr", c_vp), ("workspace", c_vp), ("vmap", c_vp), ("rlen", c_vp)]


DIA_MAX = 64


class DiaSizes(ctypes.Structure):
    _fields_ = [("n_rows", c_i64), ("n_cols", c_i64), ("n_diags", c_i32), ("offsets", c_i32 * DIA_MAX),
                ("nnz_dia", c_i64), ("nnz_rem", c_i64)]


class TransposeBuffers(ctypes.Structure):
    _fields_ = [("t_row_ptr", c_vp), ("t_col", c_vp), ("t_val", c_vp), ("tmap", c_vp),
                ("workspace", c_vp)]


class BatchItem(ctypes.Structure):
    _fields_ = [("A", c_vp), ("k", c_i32), ("X", c_vp), ("ldx", c_i64), ("Y", c_vp),
                ("ldy", c_i64)]


P = ctypes.POINTER

# name -> (restype, argtypes)
SIGNATURES = {
    "gbsp_status_string": (ctypes.c_char_p, [c_i32]),
    "gbsp_last_error": (ctypes.c_char_p, []),
    "gbsp_version": (c_i32, []),
    "gbsp_destroy": (c_i32, [c_vp]),
    "gbsp_read_status": (c_i32, [c_vp, c_vp, P(c_i32)]),
    "gbsp_set_status_word": (c_i32, [c_vp, c_vp]),
    "gbsp_crs_create": (c_i32, [c_i64, c_i64, c_i64, c_vp, c_vp, c_vp, c_i32, P(c_vp)]),
    "gbsp_crs_validate": (c_i32, [c_vp, c_vp, c_vp]),
    "gbsp_set_values": (c_i32, [c_vp, c_vp]),
    "gbsp_jds_values": (c_i32, [c_vp, c_vp, c_vp]),
    "gbsp_set_kernel": (c_i32, [c_vp, P(KernelOpts)]),
    "gbsp_get_kernel": (c_i32, [c_vp, P(KernelOpts)]),
    "gbsp_crs_tile_bytes": (c_i32, [c_vp, c_i32, P(c_i64)]),
    "gbsp_crs_prepare": (c_i32, [c_vp, c_i32, c_vp, c_i64, c_vp]),
    "gbsp_jds_plan": (c_i32, [c_vp, P(JdsOpts), c_vp, c_vp, P(JdsSizes)]),
    "gbsp_jds_build": (c_i32, [c_vp, P(JdsOpts), P(JdsBuffers), P(JdsSizes), c_vp, P(c_vp)]),
    "gbsp_jds_set_format": (c_i32, [c_vp, c_i32, c_i32, c_i32]),
    "gbsp_jds_info": (c_i32, [c_vp, P(JdsSizes), P(JdsOpts)]),
    "gbsp_jds_split_bytes": (c_i32, [c_vp, c_i32, c_i32, P(c_i64)]),
    "gbsp_jds_split": (c_i32, [c_vp, c_i32, c_i32, c_vp, c_i64, c_vp]),
    "gbsp_permute_vec": (c_i32, [c_vp, c_i32, c_i32, c_vp, c_i64, c_vp, c_i64, c_vp]),
    "gbsp_spmv": (c_i32, [c_vp, c_i32, c_i32, c_i32, c_vp, c_vp, c_vp]),
    "gbsp_spmv_host": (c_i32, [c_vp, c_i32, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "gbsp_spmm": (c_i32, [c_vp, c_i32, c_i32, c_i32, c_vp, c_i64, c_vp, c_i64, c_i32, c_vp]),
    "gbsp_transpose_workspace": (c_i32, [c_vp, P(c_i64)]),
    "gbsp_transpose_build": (c_i32, [c_vp, P(TransposeBuffers), c_i64, c_vp, P(c_vp)]),
    "gbsp_transpose_values": (c_i32, [c_vp, c_vp]),
    "gbsp_attach_transpose": (c_i32, [c_vp, c_vp]),
    "gbsp_dval": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i32, c_vp]),
    "gbsp_dval_multi": (c_i32, [c_vp, c_i32, c_vp, c_i64, c_vp, c_i64, c_vp, c_i32, c_vp]),
    "gbsp_dval_multi_strided": (c_i32, [c_vp, c_i32, c_vp, c_i64, c_i64, c_vp, c_i64, c_i64, c_vp, c_i32, c_vp]),
    "gbsp_batch_plan": (c_i32, [c_i32, P(BatchItem), c_i32, P(c_i64)]),
    "gbsp_batch_create": (c_i32, [c_i32, P(BatchItem), c_i32, c_vp, c_i64, c_vp, c_vp, P(c_vp)]),
    "gbsp_batch_run": (c_i32, [c_vp, c_vp, c_vp]),
    "gbsp_batch_info": (c_i32, [c_vp, P(c_i64), P(c_i32)]),
    "gbsp_batch_destroy": (c_i32, [c_vp]),
    "gbsp_autotune": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp, P(KernelOpts), P(c_f32)]),
    "gbsp_crs_spmv_noalloc": (c_i32, [c_i64, c_i64, c_i64, c_vp, c_vp, c_vp, c_i32, c_i32, c_vp, c_vp,
                                      c_vp]),
    "gbsp_gather_partials": (c_i32, [c_i64, ctypes.POINTER(c_i32)]),
    "gbsp_stride_hist": (c_i32, [c_vp, c_i64, c_vp, c_vp]),
    "gbsp_set_grid_limit": (c_i32, [c_vp, c_i32]),
    "gbsp_sell_stage_bytes": (c_i32, [c_vp, c_i32, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64),
                                      ctypes.POINTER(c_i64)]),
    "gbsp_sell_stage": (c_i32, [c_vp, c_i32, c_i32, c_vp, c_vp, c_vp, c_i64, c_vp]),
    "gbsp_dia_plan_workspace": (c_i32, [c_vp, ctypes.POINTER(c_i64)]),
    "gbsp_dia_plan": (c_i32, [c_vp, c_i32, ctypes.c_double, c_vp, c_vp, c_i64, c_vp, ctypes.POINTER(DiaSizes)]),
    "gbsp_dia_build": (c_i32, [c_vp, ctypes.POINTER(DiaSizes), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                               ctypes.POINTER(c_vp), ctypes.POINTER(c_vp)]),
    "gbsp_upper_workspace": (c_i32, [c_i64, ctypes.POINTER(c_i64)]),
    "gbsp_upper_plan": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_vp, ctypes.POINTER(c_i64)]),
    "gbsp_upper_build": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, c_vp, ctypes.POINTER(c_vp)]),
    "gbsp_spmv_symmetric": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_vp]),
    "gbsp_warp_sectors": (c_i32, [c_vp, c_i32, c_i32, c_vp, c_vp]),
    "gbsp_stage_sweep": (c_i32, [c_vp, c_i64, c_vp, c_i32, c_vp, c_vp]),
    "gbsp_fma_chain": (c_i32, [c_i64, c_i32, c_i32, c_vp, c_vp, c_vp]),
    "gbsp_gather_sum": (c_i32, [c_i32, c_i32, c_i64, c_i64, c_vp, c_vp, c_i64, c_vp, c_vp, c_i32, c_vp,
                                c_vp, c_vp]),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libgbspmv.so and attach the signatures (once)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build it with paper_0910_4836_gb300.build() "
                "(the CUDA library is required; there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class GbspError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


def check(status: int, what: str) -> None:
    if status != GBSP_OK:
        detail = load().gbsp_last_error().decode(errors="replace")
        raise GbspError(status, what, detail)
