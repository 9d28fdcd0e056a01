"""ctypes binding of librgcsr.so: the C structs of include/rgcsr.h and the
exported functions under the same names.  Argument marshalling only; every
computation runs in the library's CUDA kernels.  Loading fails loudly when
the library has not been built -- there is no fallback path."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

I32, I64, P, SZ = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t

RGCSR_OK = 0
RGCSR_ERR_INVALID_ARG = -1
RGCSR_ERR_BAD_ROWPTR = -2
RGCSR_ERR_COL_OOB = -3
RGCSR_ERR_INDEX_OVERFLOW = -4
RGCSR_ERR_UNSUPPORTED_DTYPE = -5
RGCSR_ERR_CUDA = -6
RGCSR_ERR_WORKSPACE = -7
RGCSR_ERR_BAD_PERM = -8
RGCSR_ERR_CORRUPT = -9
RGCSR_ERR_TIMEOUT = -10

F64, F32, BF16, F16, I32T, I64T = 0, 1, 2, 3, 4, 5

KERNEL_AUTO, KERNEL_PAPER, KERNEL_SPLIT, KERNEL_TMA, KERNEL_LEAN, KERNEL_SELL = 0, 1, 2, 3, 4, 5
STATUS_TIMEOUT, STATUS_CORRUPT = 1, 2
CHECK_GROUP_PTR, CHECK_ROW_LENGTHS, CHECK_COLUMN, CHECK_PADDING = 1, 2, 4, 8
CHECK_PERM, CHECK_SCALE, CHECK_SLOT_MAP = 16, 32, 64
XLOAD_NC, XLOAD_PLAIN, XLOAD_TEX = 0, 1, 2
XWINDOW_ROWS, XWINDOW_MAX_RANGES, XWINDOW_GAP, XWINDOW_CAP_BYTES = 256, 4, 64, 32768
VALUES_STATE_BYTES = 16384


class CSR(ctypes.Structure):
    _fields_ = [("n_rows", I64), ("n_cols", I64), ("nnz", I64),
                ("row_ptr", P), ("row_ptr_type", I32), ("value_type", I32),
                ("col_idx", P), ("values", P)]


class Matrix(ctypes.Structure):
    _fields_ = [("n_rows", I64), ("n_cols", I64), ("nnz", I64),
                ("group_size", I32), ("value_type", I32),
                ("n_groups", I64), ("n_stored", I64), ("max_row_len", I64),
                ("values", P), ("columns", P), ("group_ptr", P), ("row_lengths", P),
                ("row_scale", P), ("slot_to_csr", P), ("row_perm", P)]


class Launch(ctypes.Structure):
    _fields_ = [("kernel", I32), ("block_threads", I32), ("x_load", I32), ("split_weight", I32),
                ("variant", I32), ("wait_limit", I32)]


class Hyb(ctypes.Structure):
    _fields_ = [("n_rows", I64), ("n_cols", I64), ("nnz", I64),
                ("value_type", I32), ("ell_width", I32), ("nnz_coo", I64), ("max_row_len", I64),
                ("ell_val", P), ("ell_col", P), ("coo_row", P), ("coo_col", P), ("coo_val", P)]


class LongRows(ctypes.Structure):
    _fields_ = [("threshold", I32), ("segment", I32), ("n_segments", I64), ("n_long_rows", I64),
                ("seg_row", P), ("seg_start", P), ("long_row", P), ("long_first", P), ("long_count", P),
                ("partials", P), ("arrivals", P)]


class Tiles(ctypes.Structure):
    _fields_ = [("tile", I32), ("variant", I32), ("n_groups", I64), ("n_extra", I64), ("n_split", I64),
                ("n_partials", I64), ("first_extra", P), ("part_base", P), ("extra_group", P),
                ("arrivals", P), ("partials", P)]


class XWindow(ctypes.Structure):
    _fields_ = [("n_ranges", I32), ("total", I32), ("lo", I32 * 4), ("len", I32 * 4)]


class CheckReport(ctypes.Structure):
    _fields_ = [("flags", I32), ("reserved", I32), ("group", I64), ("row", I64), ("slot", I64)]


class BatchDesc(ctypes.Structure):
    _fields_ = [("n_rows", I64), ("n_cols", I64), ("val_off", I64), ("row_off", I64),
                ("group_off", I64), ("x_off", I64), ("group_size", I32), ("reserved", I32)]


class Batch(ctypes.Structure):
    _fields_ = [("n_matrices", I32), ("value_type", I32), ("n_tasks", I64), ("desc", P), ("tasks", P),
                ("values", P), ("columns", P), ("group_ptr", P), ("row_lengths", P), ("row_scale", P)]


_PCSR, _PM, _PL, _PH = (ctypes.POINTER(CSR), ctypes.POINTER(Matrix),
                        ctypes.POINTER(Launch), ctypes.POINTER(Hyb))
_PBD, _PB = ctypes.POINTER(BatchDesc), ctypes.POINTER(Batch)
D = ctypes.c_double
PI32, PD = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); mirrors include/rgcsr.h
SIGNATURES = {
    "rgcsr_plan_workspace_bytes": (SZ, [I64, I32]),
    "rgcsr_plan": (ctypes.c_int, [_PCSR, _PM, P, SZ, P]),
    "rgcsr_convert": (ctypes.c_int, [_PCSR, _PM, P]),
    "rgcsr_plan_noalloc": (ctypes.c_int, [_PCSR, _PM, P]),
    "rgcsr_row_order_workspace_bytes": (SZ, [I64]),
    "rgcsr_descending_order": (ctypes.c_int, [_PCSR, P, P, SZ, P]),
    "rgcsr_spmv": (ctypes.c_int, [_PM, P, P, P]),
    "rgcsr_spmv_ex": (ctypes.c_int, [_PM, P, P, _PL, P]),
    "rgcsr_auto_kernel": (ctypes.c_int, [_PM, PI32, PI32]),
    "rgcsr_spmv_host": (ctypes.c_int, [_PM, P, P, P, P, _PL, ctypes.POINTER(LongRows),
                                       ctypes.POINTER(Tiles), P]),
    "rgcsr_tiles_workspace_bytes": (SZ, [I64]),
    "rgcsr_tiles_plan": (ctypes.c_int, [_PM, ctypes.POINTER(Tiles), P, SZ, P]),
    "rgcsr_tiles_build": (ctypes.c_int, [_PM, ctypes.POINTER(Tiles), P]),
    "rgcsr_spmv_tiles": (ctypes.c_int, [_PM, ctypes.POINTER(Tiles), P, P, P]),
    "rgcsr_quantize": (ctypes.c_int, [_PM, _PM, P]),
    "rgcsr_xwindow_count": (I64, [I64]),
    "rgcsr_xwindow_plan": (ctypes.c_int, [_PM, P, P]),
    "rgcsr_spmv_xwindow": (ctypes.c_int, [_PM, P, P, P, P]),
    "rgcsr_long_rows_workspace_bytes": (SZ, [I64]),
    "rgcsr_long_rows_plan": (ctypes.c_int, [_PM, ctypes.POINTER(LongRows), P, SZ, P]),
    "rgcsr_long_rows_build": (ctypes.c_int, [_PM, ctypes.POINTER(LongRows), P, SZ, P]),
    "rgcsr_spmv_long_rows": (ctypes.c_int, [_PM, ctypes.POINTER(LongRows), P, P, P]),
    "rgcsr_spmm": (ctypes.c_int, [_PM, I32, P, I64, P, I64, P]),
    "rgcsr_spmm_long_rows": (ctypes.c_int, [_PM, ctypes.POINTER(LongRows), I32, P, I64, P, I64, P, I64, P]),
    "rgcsr_spmm_tiles": (ctypes.c_int, [_PM, ctypes.POINTER(Tiles), I32, P, I64, P, I64, P, I64, P]),
    "rgcsr_transpose_workspace_bytes": (SZ, [I64, I64, I64]),
    "rgcsr_csr_transpose": (ctypes.c_int, [_PCSR, P, P, P, P, P, SZ, P]),
    "rgcsr_csr_row_index": (ctypes.c_int, [_PCSR, P, P]),
    "rgcsr_gather_values": (ctypes.c_int, [_PM, P, P, P]),
    "rgcsr_gather_values_if_changed": (ctypes.c_int, [_PM, P, I64, P, P, P]),
    "rgcsr_compose_index": (ctypes.c_int, [P, P, I64, P, P]),
    "rgcsr_sampled_dot": (ctypes.c_int, [I64, I32, P, P, P, I64, P, I64, P, I32, P]),
    "rgcsr_spmv_bwd_values": (ctypes.c_int, [_PM, I32, P, I64, P, I64, P, P]),
    "rgcsr_batch_tasks": (ctypes.c_int, [_PBD, I32, P, I64, ctypes.POINTER(I64)]),
    "rgcsr_spmv_batched": (ctypes.c_int, [_PB, P, P, P]),
    "rgcsr_dot_workspace_bytes": (SZ, []),
    "rgcsr_dot": (ctypes.c_int, [I64, P, P, P, P, SZ, I32, P]),
    "rgcsr_axpby": (ctypes.c_int, [I64, D, P, D, P, I32, P]),
    "rgcsr_jacobi_step": (ctypes.c_int, [I64, D, P, P, P, P, P, I32, P]),
    "rgcsr_diag_scale": (ctypes.c_int, [I64, D, P, P, P, I32, P]),
    "rgcsr_convert_vector": (ctypes.c_int, [I64, P, I32, P, I32, P]),
    "rgcsr_stream_read": (ctypes.c_int, [P, I64, P, P]),
    "rgcsr_fp64_fma_probe": (ctypes.c_int, [I32, P, ctypes.POINTER(I64), P]),
    "rgcsr_gather_probe": (ctypes.c_int, [P, I64, I32, P, ctypes.POINTER(I64), P]),
    "rgcsr_cg_workspace_bytes": (SZ, [I64, I32]),
    "rgcsr_cg": (ctypes.c_int, [_PM, P, P, D, I32, I32, P, SZ, PI32, PD, P]),
    "rgcsr_ir_cg_workspace_bytes": (SZ, [I64]),
    "rgcsr_ir_cg": (ctypes.c_int, [_PM, _PM, P, P, D, I32, D, I32, P, SZ, PI32, PI32, PD, P]),
    "hyb_workspace_bytes": (SZ, [I64, I64]),
    "hyb_plan": (ctypes.c_int, [_PCSR, I32, _PH, P, SZ, P]),
    "hyb_convert": (ctypes.c_int, [_PCSR, _PH, P, SZ, P]),
    "hyb_spmv": (ctypes.c_int, [_PH, P, P, P]),
    "hyb_spmm": (ctypes.c_int, [_PH, I32, P, I64, P, I64, P]),
    "rgcsr_check_matrix": (ctypes.c_int, [_PM, ctypes.POINTER(CheckReport), P]),
    "rgcsr_set_checks": (ctypes.c_int, [ctypes.c_int]),
    "rgcsr_set_wait_limit": (ctypes.c_int, [I32]),
    "rgcsr_get_status": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), P]),
    "rgcsr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "rgcsr_version": (ctypes.c_int, []),
}

_lib = None


class RgCSRError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        msg = lib().rgcsr_status_string(status).decode()
        super().__init__(f"{fn} failed: {msg} ({status})")


def lib():
    """The loaded library.  Raises if librgcsr.so was not built."""
    global _lib
    if _lib is None:
        path = _build.LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(
                f"librgcsr.so not found at {path}; build it first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def call(name: str, *args) -> int:
    """Call an exported function; raise RgCSRError on a negative status."""
    st = getattr(lib(), name)(*args)
    if st != RGCSR_OK:
        raise RgCSRError(name, st)
    return st
