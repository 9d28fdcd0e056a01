"""Row-grouped CSR (RgCSR) and Hybrid ELL+COO matrices on the GPU.

PyTorch provides device memory and streams only: every array is a torch
tensor that this module allocates from the sizes the library's ``*_plan``
calls return, and every computation (validation, conversion, SpMV) is a
call into librgcsr's CUDA kernels on the current torch stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L

_VT = {torch.float64: L.F64, torch.float32: L.F32}


# rgcsr_check_matrix's checks: (name, RGCSR_CHECK_* bit)
CHECKS = (("group_ptr", L.CHECK_GROUP_PTR), ("row_lengths", L.CHECK_ROW_LENGTHS), ("column", L.CHECK_COLUMN),
          ("padding", L.CHECK_PADDING), ("perm", L.CHECK_PERM), ("scale", L.CHECK_SCALE),
          ("slot_map", L.CHECK_SLOT_MAP))


def set_checks(on: bool) -> bool:
    """Checks mode (rgcsr_set_checks): every product checks its matrix
    first and refuses a corrupt one.  Returns the previous setting."""
    return bool(L.lib().rgcsr_set_checks(1 if on else 0))


def get_status(stream=None) -> int:
    """The library's sticky status bits (rgcsr_get_status), cleared by the read."""
    st = ctypes.c_int(0)
    L.call("rgcsr_get_status", ctypes.byref(st), _stream_ptr(stream))
    return st.value


def _stream_ptr(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr() if t is not None and t.numel() > 0 else 0)


def stream_read(buf: torch.Tensor, stream=None) -> None:
    """Reads the bytes of `buf` (contiguous, CUDA, a multiple of 16 bytes)
    with the library's plain streaming-read kernel: the bandwidth reference
    for a memory-bound kernel that moves as many bytes."""
    if not (buf.is_cuda and buf.is_contiguous()):
        raise ValueError("stream_read needs a contiguous CUDA tensor")
    sink = _READ_SINKS.get(buf.device)
    if sink is None:                 # allocated once, so a timed call launches only the read
        sink = _READ_SINKS[buf.device] = torch.zeros(1, dtype=torch.float32, device=buf.device)
    L.call("rgcsr_stream_read", _ptr(buf), buf.numel() * buf.element_size(), _ptr(sink), _stream_ptr(stream))


_READ_SINKS: dict = {}


def fp64_fma_probe(iters: int = 1024, stream=None) -> int:
    """Launches the library's FP64 FMA throughput kernel (independent FMA
    chains on every SM) and returns how many FMAs it runs."""
    dev = torch.device("cuda", torch.cuda.current_device())
    sink = _FMA_SINKS.get(dev)
    if sink is None:
        sink = _FMA_SINKS[dev] = torch.zeros(1, dtype=torch.float64, device=dev)
    n = ctypes.c_int64(0)
    L.call("rgcsr_fp64_fma_probe", int(iters), _ptr(sink), ctypes.byref(n), _stream_ptr(stream))
    return n.value


_FMA_SINKS: dict = {}


def gather_probe(x: torch.Tensor, iters: int = 256, stream=None) -> int:
    """Launches the library's random-gather kernel over the double vector x
    (length a power of two) and returns how many 8-byte loads it issues."""
    if not (x.is_cuda and x.is_contiguous() and x.dtype == torch.float64):
        raise ValueError("gather_probe needs a contiguous CUDA float64 tensor")
    sink = _FMA_SINKS.get(x.device)
    if sink is None:
        sink = _FMA_SINKS[x.device] = torch.zeros(1, dtype=torch.float64, device=x.device)
    n = ctypes.c_int64(0)
    L.call("rgcsr_gather_probe", _ptr(x), x.numel(), int(iters), _ptr(sink), ctypes.byref(n), _stream_ptr(stream))
    return n.value


def _dev(a, dtype=None, device="cuda") -> torch.Tensor:
    t = torch.as_tensor(np.ascontiguousarray(a)) if isinstance(a, np.ndarray) else a
    if dtype is not None and t.dtype != dtype:
        t = t.to(dtype)
    return t.to(device).contiguous()


def csr_struct(rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, n_cols: int) -> L.CSR:
    if rowptr.dtype not in (torch.int32, torch.int64):
        raise TypeError("row pointer must be int32 or int64")
    if col.dtype != torch.int32:
        raise TypeError("column indices must be int32")
    if val.dtype not in _VT:
        raise TypeError("values must be float32 or float64")
    c = L.CSR()
    c.n_rows = rowptr.numel() - 1
    c.n_cols = int(n_cols)
    c.nnz = col.numel()
    c.row_ptr = _ptr(rowptr)
    c.row_ptr_type = L.I64T if rowptr.dtype == torch.int64 else L.I32T
    c.value_type = _VT[val.dtype]
    c.col_idx = _ptr(col)
    c.values = _ptr(val)
    return c


class RgCSRMatrix:
    """A matrix in Row-grouped CSR (Sec. 3.4 of the paper) on one GPU.

    Attributes are torch tensors: ``values`` [n_stored], ``columns`` int32
    [n_stored], ``group_ptr`` int64 [n_groups+1], ``row_lengths`` int32
    [n_rows] and optionally ``slot_to_csr`` int64 [n_stored] and
    ``row_perm`` int32 [n_rows] (the CSR row held by each stored row when a
    row order was used; x and y are always in the CSR's row order).
    """

    def __init__(self):
        self.s = L.Matrix()
        self.values = self.columns = self.group_ptr = self.row_lengths = None
        self.row_scale = None
        self.slot_to_csr = None
        self.row_perm = None
        self._long = None          # long-row segment schedule, if enabled
        self._tiles = None         # group-tile schedule, if enabled
        self._xwin = None          # shared-memory x windows, if planned

    # -- construction ------------------------------------------------------
    @classmethod
    def from_csr(cls, rowptr, col, val, n_cols: int, group_size: int = 32,
                 dtype: torch.dtype | None = None, keep_slot_map: bool = False,
                 row_order=None, device="cuda", stream=None) -> "RgCSRMatrix":
        """Converts a CSR matrix (host numpy or device tensors) to RgCSR.

        ``dtype`` (float32/float64) is the storage type of the values; the
        CSR values are cast to it before conversion.  ``row_order``: None
        (rows in CSR order), "descending" (rows by length, longest first,
        stable -- Sec. 4.4.2, Table 7), or any permutation of the rows as an
        int32 array (stored row k = CSR row row_order[k]).  Synchronises
        once."""
        rowptr = _dev(rowptr, None, device)
        col = _dev(col, torch.int32, device)
        val = _dev(val, dtype, device)
        A = csr_struct(rowptr, col, val, n_cols)
        self = cls()
        n = A.n_rows
        G = int(group_size)
        if G < 1:
            raise ValueError("group_size must be >= 1")
        n_groups = (n + G - 1) // G
        self.row_lengths = torch.empty(n, dtype=torch.int32, device=device)
        self.group_ptr = torch.empty(n_groups + 1, dtype=torch.int64, device=device)
        M = self.s
        M.group_size = G
        M.value_type = A.value_type
        M.row_lengths = _ptr(self.row_lengths)
        M.group_ptr = _ptr(self.group_ptr)
        st = _stream_ptr(stream)
        if row_order is not None and n > 0:
            if isinstance(row_order, str):
                if row_order != "descending":
                    raise ValueError(f"unknown row order {row_order!r}")
                self.row_perm = torch.empty(n, dtype=torch.int32, device=device)
                ob = L.lib().rgcsr_row_order_workspace_bytes(n)
                ows = torch.empty(ob, dtype=torch.uint8, device=device)
                L.call("rgcsr_descending_order", ctypes.byref(A), _ptr(self.row_perm), _ptr(ows), ob, st)
            else:
                self.row_perm = _dev(row_order, torch.int32, device)
                if self.row_perm.numel() != n:
                    raise ValueError("row_order must have one entry per row")
            M.row_perm = _ptr(self.row_perm)
        ws_bytes = L.lib().rgcsr_plan_workspace_bytes(n, G)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=device)
        L.call("rgcsr_plan", ctypes.byref(A), ctypes.byref(M), _ptr(ws), ws_bytes, st)
        self.values = torch.empty(M.n_stored, dtype=val.dtype, device=device)
        self.columns = torch.empty(M.n_stored, dtype=torch.int32, device=device)
        M.values = _ptr(self.values)
        M.columns = _ptr(self.columns)
        if keep_slot_map:
            self.slot_to_csr = torch.empty(M.n_stored, dtype=torch.int64, device=device)
            M.slot_to_csr = _ptr(self.slot_to_csr)
        L.call("rgcsr_convert", ctypes.byref(A), ctypes.byref(M), st)
        return self

    def split_long_rows(self, threshold: int = 64, segment: int = 256, stream=None) -> "RgCSRMatrix":
        """Makes spmv() cut the slots >= threshold of longer rows into
        segments of `segment` slots, one warp each (rgcsr_spmv_long_rows).
        The schedule's partial sums and arrival counters are the product's
        scratch, so one product per schedule may be in flight at a time:
        products on several streams need a matrix (or schedule) each."""
        S = L.LongRows()
        S.threshold, S.segment = int(threshold), int(segment)
        dev = self.group_ptr.device
        nb = L.lib().rgcsr_long_rows_workspace_bytes(self.s.n_rows)
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        st = _stream_ptr(stream)
        L.call("rgcsr_long_rows_plan", ctypes.byref(self.s), ctypes.byref(S), _ptr(ws), nb, st)
        i32 = dict(dtype=torch.int32, device=dev)
        bufs = dict(seg_row=torch.empty(S.n_segments, **i32), seg_start=torch.empty(S.n_segments, **i32),
                    long_row=torch.empty(S.n_long_rows, **i32), long_first=torch.empty(S.n_long_rows, **i32),
                    long_count=torch.empty(S.n_long_rows, **i32), arrivals=torch.empty(S.n_segments, **i32),
                    partials=torch.empty(S.n_segments, dtype=self.x_dtype, device=dev))
        for k, t in bufs.items():
            setattr(S, k, _ptr(t))
        L.call("rgcsr_long_rows_build", ctypes.byref(self.s), ctypes.byref(S), _ptr(ws), nb, st)
        self._long = (S, bufs)
        return self

    def tile_groups(self, tile: int = 64, variant: int = 0, stream=None) -> "RgCSRMatrix":
        """Makes spmv() use the group-tile schedule (rgcsr_spmv_tiles): one
        warp per tile of at most `tile` slot-rows of a group, long groups cut
        into several tiles.  Needs group_size <= 32.  As with the long-row
        schedule, one product per schedule may be in flight at a time."""
        T = L.Tiles()
        T.tile = int(tile)
        T.variant = int(variant)
        dev = self.group_ptr.device
        ng = self.s.n_groups
        i64 = dict(dtype=torch.int64, device=dev)
        bufs = dict(first_extra=torch.empty(ng + 1, **i64), part_base=torch.empty(ng + 1, **i64))
        T.first_extra, T.part_base = _ptr(bufs["first_extra"]), _ptr(bufs["part_base"])
        nb = L.lib().rgcsr_tiles_workspace_bytes(ng)
        ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=dev)
        st = _stream_ptr(stream)
        L.call("rgcsr_tiles_plan", ctypes.byref(self.s), ctypes.byref(T), _ptr(ws), nb, st)
        bufs["extra_group"] = torch.empty(T.n_extra, dtype=torch.int32, device=dev)
        bufs["arrivals"] = torch.empty(ng if T.n_extra else 0, dtype=torch.int32, device=dev)
        bufs["partials"] = torch.empty(T.n_partials * 32, dtype=self.x_dtype, device=dev)
        for k in ("extra_group", "arrivals", "partials"):
            setattr(T, k, _ptr(bufs[k]))
        L.call("rgcsr_tiles_build", ctypes.byref(self.s), ctypes.byref(T), st)
        self._tiles = (T, bufs)
        return self

    def copy_schedule(self, other: "RgCSRMatrix") -> "RgCSRMatrix":
        """Builds the same launch schedule (tiles or long-row segments) as
        `other`, a matrix with the same layout (e.g. its quantised copy)."""
        self._long = self._tiles = None
        if other._tiles is not None:
            self.tile_groups(other._tiles[0].tile, other._tiles[0].variant)
        elif other._long is not None:
            self.split_long_rows(other._long[0].threshold, other._long[0].segment)
        return self

    def auto_kernel(self) -> tuple:
        """(kernel, variant) that spmv() runs without a schedule or options
        (rgcsr_auto_kernel: the library's RGCSR_KERNEL_AUTO rule)."""
        k, v = ctypes.c_int32(0), ctypes.c_int32(0)
        L.call("rgcsr_auto_kernel", ctypes.byref(self.s), ctypes.byref(k), ctypes.byref(v))
        return k.value, v.value

    def check(self, stream=None) -> dict:
        """The library's structural checks of the stored layout
        (rgcsr_check_matrix): {"ok", "flags" (names of the failed checks),
        "group", "row", "slot" (the lowest failing ones, -1 = none)}."""
        rep = L.CheckReport()
        st = L.lib().rgcsr_check_matrix(ctypes.byref(self.s), ctypes.byref(rep), _stream_ptr(stream))
        if st not in (L.RGCSR_OK, L.RGCSR_ERR_CORRUPT):
            raise L.RgCSRError("rgcsr_check_matrix", st)
        return {"ok": st == L.RGCSR_OK, "flags": [n for n, b in CHECKS if rep.flags & b],
                "group": rep.group, "row": rep.row, "slot": rep.slot}

    def plan_x_window(self, stream=None) -> "RgCSRMatrix":
        """Plans the shared-memory x window of every block of 256 stored rows
        (rgcsr_xwindow_plan) for spmv_xwindow()."""
        nb = L.lib().rgcsr_xwindow_count(self.s.n_rows)
        self._xwin = torch.empty(max(nb, 1) * ctypes.sizeof(L.XWindow), dtype=torch.uint8,
                                 device=self.group_ptr.device)
        L.call("rgcsr_xwindow_plan", ctypes.byref(self.s), _ptr(self._xwin), _stream_ptr(stream))
        return self

    def x_window_records(self) -> list:
        """The planned windows as (n_ranges, total, lo, len) per block (host copy)."""
        raw = self._xwin.cpu().numpy().view(np.int32).reshape(-1, 10)
        nb = L.lib().rgcsr_xwindow_count(self.s.n_rows)
        return [(int(r[0]), int(r[1]), r[2:6].tolist(), r[6:10].tolist()) for r in raw[:nb]]

    def spmv_xwindow(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """y = A x with each planned block's x ranges staged in shared memory."""
        if getattr(self, "_xwin", None) is None:
            raise ValueError("call plan_x_window() first")
        if x.dtype != self.x_dtype or x.numel() != self.s.n_cols or not x.is_contiguous():
            raise ValueError(f"x must be a contiguous {self.x_dtype} vector of length {self.s.n_cols}")
        y = out if out is not None else torch.empty(self.s.n_rows, dtype=self.x_dtype, device=x.device)
        L.call("rgcsr_spmv_xwindow", ctypes.byref(self.s), _ptr(self._xwin), _ptr(x), _ptr(y),
               _stream_ptr(stream))
        return y

    @property
    def n_extra_tiles(self) -> int:
        return 0 if self._tiles is None else self._tiles[0].n_extra

    @property
    def n_long_segments(self) -> int:
        return 0 if self._long is None else self._long[0].n_segments

    def quantized(self, fmt: str = "bf16", stream=None) -> "RgCSRMatrix":
        """The same matrix with values stored as bfloat16 ("bf16") or half
        ("f16") and a per-row power-of-two float scale; shares columns, group
        pointers and row lengths with this matrix."""
        q = RgCSRMatrix()
        q.columns, q.group_ptr, q.row_lengths = self.columns, self.group_ptr, self.row_lengths
        q.slot_to_csr = self.slot_to_csr
        q.row_perm = self.row_perm
        dt = {"bf16": torch.bfloat16, "f16": torch.float16}[fmt]
        dev = self.group_ptr.device
        q.values = torch.empty(self.s.n_stored, dtype=dt, device=dev)
        q.row_scale = torch.empty(self.s.n_rows, dtype=torch.float32, device=dev)
        D = q.s
        D.value_type = L.BF16 if fmt == "bf16" else L.F16
        D.values, D.row_scale = _ptr(q.values), _ptr(q.row_scale)
        D.columns, D.group_ptr, D.row_lengths = self.s.columns, self.s.group_ptr, self.s.row_lengths
        D.slot_to_csr = self.s.slot_to_csr
        L.call("rgcsr_quantize", ctypes.byref(self.s), ctypes.byref(D), _stream_ptr(stream))
        return q

    # -- properties ----------------------------------------------------------
    @property
    def shape(self):
        return (self.s.n_rows, self.s.n_cols)

    @property
    def nnz(self) -> int:
        return self.s.nnz

    @property
    def n_stored(self) -> int:
        return self.s.n_stored

    @property
    def group_size(self) -> int:
        return self.s.group_size

    @property
    def max_row_len(self) -> int:
        return self.s.max_row_len

    @property
    def dtype(self) -> torch.dtype:
        return self.values.dtype

    @property
    def x_dtype(self) -> torch.dtype:
        return torch.float64 if self.s.value_type == L.F64 else torch.float32

    def artificial_zero_percent(self) -> float:
        return 100.0 * (self.n_stored - self.nnz) / self.nnz if self.nnz else 0.0

    # -- products --------------------------------------------------------------
    def spmv(self, x: torch.Tensor, out: torch.Tensor | None = None,
             kernel: int = L.KERNEL_AUTO, x_load: int = L.XLOAD_NC, block_threads: int = 0,
             split_weight: int = 0, variant: int = 0, wait_limit: int = 0, stream=None) -> torch.Tensor:
        """y = A x (overwrites ``out`` if given).  wait_limit: probes before a
        bounded wait of the TMA kernel gives up (0 = the library's default;
        small values only to exercise the timeout path)."""
        if x.dtype != self.x_dtype or x.numel() != self.s.n_cols or not x.is_contiguous():
            raise ValueError(f"x must be a contiguous {self.x_dtype} vector of length {self.s.n_cols}")
        y = out if out is not None else torch.empty(self.s.n_rows, dtype=self.x_dtype, device=x.device)
        default = (kernel == L.KERNEL_AUTO and x_load == L.XLOAD_NC and not block_threads
                   and not split_weight and not variant and not wait_limit)
        if default and self._tiles is not None:
            L.call("rgcsr_spmv_tiles", ctypes.byref(self.s), ctypes.byref(self._tiles[0]), _ptr(x), _ptr(y),
                   _stream_ptr(stream))
        elif default and self._long is not None:
            L.call("rgcsr_spmv_long_rows", ctypes.byref(self.s), ctypes.byref(self._long[0]), _ptr(x), _ptr(y),
                   _stream_ptr(stream))
        elif default:
            L.call("rgcsr_spmv", ctypes.byref(self.s), _ptr(x), _ptr(y), _stream_ptr(stream))
        else:
            ln = L.Launch(kernel, block_threads, x_load, split_weight, variant, wait_limit)
            L.call("rgcsr_spmv_ex", ctypes.byref(self.s), _ptr(x), _ptr(y), ctypes.byref(ln),
                   _stream_ptr(stream))
        return y

    def spmm(self, X: torch.Tensor, out: torch.Tensor | None = None, rows: bool | None = None,
             stream=None) -> torch.Tensor:
        """Y = A X for X of shape [n_cols, k] with unit column stride.

        With a group-tile schedule (tile_groups) and rows not set: the tiled
        kernels (rgcsr_spmm_tiles).  rows: the lanes-per-row kernels
        (rgcsr_spmm_long_rows), with the long-row schedule if one was built;
        the default when a long-row schedule exists.  Else rgcsr_spmm."""
        if X.dim() != 2 or X.shape[0] != self.s.n_cols or X.dtype != self.x_dtype or X.stride(1) != 1:
            raise ValueError(f"X must be [{self.s.n_cols}, k] {self.x_dtype} with unit column stride")
        k = X.shape[1]
        Y = out if out is not None else torch.empty(self.s.n_rows, k, dtype=self.x_dtype, device=X.device)
        if Y.shape != (self.s.n_rows, k) or Y.stride(1) != 1:
            raise ValueError("out must be [n_rows, k] with unit column stride")
        ldx, ldy = max(X.stride(0), k), max(Y.stride(0), k)
        if rows is None and self._tiles is not None:
            T, bufs = self._tiles
            need = T.n_partials * 32 * min(k, 8)
            if bufs.get("spmm_partials") is None or bufs["spmm_partials"].numel() < need:
                bufs["spmm_partials"] = torch.empty(max(need, 1), dtype=self.x_dtype, device=X.device)
            part = bufs["spmm_partials"]
            L.call("rgcsr_spmm_tiles", ctypes.byref(self.s), ctypes.byref(T), k, _ptr(X), ldx, _ptr(Y), ldy,
                   _ptr(part), part.numel(), _stream_ptr(stream))
            return Y
        if rows is None:
            rows = self._long is not None
        if not rows:
            L.call("rgcsr_spmm", ctypes.byref(self.s), k, _ptr(X), ldx, _ptr(Y), ldy, _stream_ptr(stream))
            return Y
        lr, part = None, None
        if self._long is not None:
            lr = ctypes.byref(self._long[0])
            need = self._long[0].n_segments * min(k, 32)
            bufs = self._long[1]
            if bufs.get("spmm_partials") is None or bufs["spmm_partials"].numel() < need:
                bufs["spmm_partials"] = torch.empty(max(need, 1), dtype=self.x_dtype, device=X.device)
            part = bufs["spmm_partials"]
        L.call("rgcsr_spmm_long_rows", ctypes.byref(self.s), lr, k, _ptr(X), ldx, _ptr(Y), ldy, _ptr(part),
               0 if part is None else part.numel(), _stream_ptr(stream))
        return Y

    def value_grad(self, Gy: torch.Tensor, X: torch.Tensor, stream=None) -> torch.Tensor:
        """d/d(values) of sum(Gy * (A X)), in the CSR's entry order:
        dval_p = sum_b Gy[row_p, b] X[col_p, b] (rgcsr_spmv_bwd_values).
        Gy [n_rows, k] and X [n_cols, k] (or vectors); needs keep_slot_map."""
        if self.slot_to_csr is None:
            raise ValueError("value_grad needs the slot map (from_csr(..., keep_slot_map=True))")
        G2, X2 = Gy.reshape(self.s.n_rows, -1), X.reshape(self.s.n_cols, -1)
        if G2.dtype != self.x_dtype or X2.dtype != self.x_dtype or G2.shape[1] != X2.shape[1]:
            raise ValueError("Gy and X must share the matrix's vector type and column count")
        if G2.stride(-1) != 1 or X2.stride(-1) != 1:
            raise ValueError("Gy and X need unit column stride")
        k = G2.shape[1]
        out = torch.empty(self.s.nnz, dtype=self.x_dtype, device=X.device)
        L.call("rgcsr_spmv_bwd_values", ctypes.byref(self.s), k, _ptr(G2), max(G2.stride(0), k), _ptr(X2),
               max(X2.stride(0), k), _ptr(out), _stream_ptr(stream))
        return out

    def spmv_host(self, x_host: torch.Tensor, y_host: torch.Tensor, x_dev: torch.Tensor,
                  y_dev: torch.Tensor, kernel: int = L.KERNEL_AUTO, variant: int = 0, stream=None) -> None:
        """Host-to-host SpMV through caller-provided device staging buffers
        (the tile or long-row schedule if enabled, else the given kernel)."""
        launch = lr = tl = None
        default = kernel == L.KERNEL_AUTO and not variant
        if default and self._tiles is not None:
            tl = ctypes.byref(self._tiles[0])
        elif default and self._long is not None:
            lr = ctypes.byref(self._long[0])
        else:
            launch = ctypes.byref(L.Launch(kernel, 0, L.XLOAD_NC, 0, variant))
        L.call("rgcsr_spmv_host", ctypes.byref(self.s), _ptr(x_host), _ptr(y_host),
               _ptr(x_dev), _ptr(y_dev), launch, lr, tl, _stream_ptr(stream))

    def __matmul__(self, x):
        return self.spmv(x)


class HybMatrix:
    """Hybrid ELLPACK + COO (Sec. 3.3 of the paper) on one GPU."""

    def __init__(self):
        self.s = L.Hyb()
        self.ell_val = self.ell_col = self.coo_row = self.coo_col = self.coo_val = None

    @classmethod
    def from_csr(cls, rowptr, col, val, n_cols: int, ell_width: int = -1,
                 dtype: torch.dtype | None = None, device="cuda", stream=None) -> "HybMatrix":
        rowptr = _dev(rowptr, None, device)
        col = _dev(col, torch.int32, device)
        val = _dev(val, dtype, device)
        A = csr_struct(rowptr, col, val, n_cols)
        self = cls()
        H = self.s
        ws_bytes = L.lib().hyb_workspace_bytes(A.n_rows, A.n_cols)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=device)
        st = _stream_ptr(stream)
        L.call("hyb_plan", ctypes.byref(A), int(ell_width), ctypes.byref(H), _ptr(ws), ws_bytes, st)
        n, K1, nc = H.n_rows, H.ell_width, H.nnz_coo
        self.ell_val = torch.empty(n * K1, dtype=val.dtype, device=device)
        self.ell_col = torch.empty(n * K1, dtype=torch.int32, device=device)
        self.coo_row = torch.empty(nc, dtype=torch.int32, device=device)
        self.coo_col = torch.empty(nc, dtype=torch.int32, device=device)
        self.coo_val = torch.empty(nc, dtype=val.dtype, device=device)
        H.ell_val, H.ell_col = _ptr(self.ell_val), _ptr(self.ell_col)
        H.coo_row, H.coo_col, H.coo_val = _ptr(self.coo_row), _ptr(self.coo_col), _ptr(self.coo_val)
        L.call("hyb_convert", ctypes.byref(A), ctypes.byref(H), _ptr(ws), ws_bytes, st)
        return self

    @property
    def shape(self):
        return (self.s.n_rows, self.s.n_cols)

    @property
    def nnz(self) -> int:
        return self.s.nnz

    @property
    def ell_width(self) -> int:
        return self.s.ell_width

    @property
    def nnz_coo(self) -> int:
        return self.s.nnz_coo

    @property
    def x_dtype(self) -> torch.dtype:
        return torch.float64 if self.s.value_type == L.F64 else torch.float32

    def spmv(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if x.dtype != self.x_dtype or x.numel() != self.s.n_cols or not x.is_contiguous():
            raise ValueError(f"x must be a contiguous {self.x_dtype} vector of length {self.s.n_cols}")
        y = out if out is not None else torch.empty(self.s.n_rows, dtype=self.x_dtype, device=x.device)
        L.call("hyb_spmv", ctypes.byref(self.s), _ptr(x), _ptr(y), _stream_ptr(stream))
        return y

    def spmm(self, X: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Y = A X for X of shape [n_cols, k] with unit column stride."""
        if X.dim() != 2 or X.shape[0] != self.s.n_cols or X.dtype != self.x_dtype or X.stride(1) != 1:
            raise ValueError(f"X must be [{self.s.n_cols}, k] {self.x_dtype} with unit column stride")
        k = X.shape[1]
        Y = out if out is not None else torch.empty(self.s.n_rows, k, dtype=self.x_dtype, device=X.device)
        if Y.shape != (self.s.n_rows, k) or Y.stride(1) != 1:
            raise ValueError("out must be [n_rows, k] with unit column stride")
        L.call("hyb_spmm", ctypes.byref(self.s), k, _ptr(X), max(X.stride(0), k), _ptr(Y), max(Y.stride(0), k),
               _stream_ptr(stream))
        return Y

    def __matmul__(self, x):
        return self.spmv(x)
