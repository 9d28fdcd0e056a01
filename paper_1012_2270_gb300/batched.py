"""Many RgCSR matrices of uneven sizes multiplied in one launch.

``BatchedRgCSR.from_csr_list`` converts every member with librgcsr's plan /
convert kernels directly into slices of shared concatenated arrays, builds
the per-member descriptors and the 32-row task list (rgcsr_batch_tasks) and
keeps everything on the GPU.  ``spmv`` is one rgcsr_spmv_batched launch;
``capture`` records it into a CUDA graph for replay.

``BlockDiagonalBatch`` is the other way to batch: the members form one
block-diagonal matrix diag(A_1, ..., A_m), so one SpMV of it with the
concatenated x computes every member's product.  Its rows can be put in
descending length order across the whole batch and its groups cut into
tiles (rgcsr_spmv_tiles), so uneven members and uneven rows share one
balanced launch.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L
from .autotune import model_group_size
from .rgcsr import _dev, _ptr, _stream_ptr, csr_struct

_VT = {torch.float64: L.F64, torch.float32: L.F32}


class BatchedRgCSR:
    def __init__(self):
        self.s = L.Batch()

    @classmethod
    def from_csr_list(cls, mats, dtype: torch.dtype = torch.float32, group_sizes="model",
                      device="cuda") -> "BatchedRgCSR":
        """``mats``: objects with rowptr, col, val, n_rows, n_cols (host
        numpy).  ``group_sizes``: "model" (per-member choice by the padding
        model), an int for all members, or a list."""
        self = cls()
        m = len(mats)
        if group_sizes == "model":
            Gs = [model_group_size(A.rowptr, dtype.itemsize) for A in mats]
        elif isinstance(group_sizes, int):
            Gs = [group_sizes] * m
        else:
            Gs = list(group_sizes)
        self.group_sizes = Gs
        n_rows = np.array([A.n_rows for A in mats], np.int64)
        n_cols = np.array([A.n_cols for A in mats], np.int64)
        n_groups = np.array([(A.n_rows + G - 1) // G for A, G in zip(mats, Gs)], np.int64)
        row_off = np.concatenate([[0], np.cumsum(n_rows)])
        x_off = np.concatenate([[0], np.cumsum(n_cols)])
        group_off = np.concatenate([[0], np.cumsum(n_groups + 1)])
        self.n_rows_total, self.n_cols_total = int(row_off[-1]), int(x_off[-1])
        self.row_lengths = torch.empty(max(self.n_rows_total, 1), dtype=torch.int32, device=device)
        self.group_ptr = torch.empty(int(group_off[-1]), dtype=torch.int64, device=device)
        st = _stream_ptr()
        lib = L.lib()
        # plan every member into its slice of row_lengths / group_ptr
        plans = []
        for i, (A, G) in enumerate(zip(mats, Gs)):
            rp, col, val = _dev(A.rowptr, None, device), _dev(A.col, torch.int32, device), _dev(A.val, dtype, device)
            csr = csr_struct(rp, col, val, A.n_cols)
            M = L.Matrix()
            M.group_size, M.value_type = G, _VT[dtype]
            M.row_lengths = ctypes.c_void_p(self.row_lengths.data_ptr() + 4 * int(row_off[i]))
            M.group_ptr = ctypes.c_void_p(self.group_ptr.data_ptr() + 8 * int(group_off[i]))
            nb = lib.rgcsr_plan_workspace_bytes(A.n_rows, G)
            ws = torch.empty(nb, dtype=torch.uint8, device=device)
            L.call("rgcsr_plan", ctypes.byref(csr), ctypes.byref(M), _ptr(ws), nb, st)
            plans.append(M)
        n_stored = np.array([M.n_stored for M in plans], np.int64)
        val_off = np.concatenate([[0], np.cumsum(n_stored)])
        self.n_stored, self.nnz = int(val_off[-1]), int(sum(A.nnz for A in mats))
        self.values = torch.empty(max(self.n_stored, 1), dtype=dtype, device=device)
        self.columns = torch.empty(max(self.n_stored, 1), dtype=torch.int32, device=device)
        for i, (A, M) in enumerate(zip(mats, plans)):
            if M.n_stored == 0:
                continue
            rp, col, val = _dev(A.rowptr, None, device), _dev(A.col, torch.int32, device), _dev(A.val, dtype, device)
            M.values = ctypes.c_void_p(self.values.data_ptr() + dtype.itemsize * int(val_off[i]))
            M.columns = ctypes.c_void_p(self.columns.data_ptr() + 4 * int(val_off[i]))
            L.call("rgcsr_convert", ctypes.byref(csr_struct(rp, col, val, A.n_cols)), ctypes.byref(M), st)
        # descriptors and tasks (host), then to the device
        descs = (L.BatchDesc * m)()
        for i in range(m):
            d = descs[i]
            d.n_rows, d.n_cols = int(n_rows[i]), int(n_cols[i])
            d.val_off, d.row_off = int(val_off[i]), int(row_off[i])
            d.group_off, d.x_off = int(group_off[i]), int(x_off[i])
            d.group_size = int(Gs[i])
        n_tasks = ctypes.c_int64(0)
        L.call("rgcsr_batch_tasks", descs, m, None, 0, ctypes.byref(n_tasks))
        tasks = np.empty(2 * max(n_tasks.value, 1), np.int32)
        L.call("rgcsr_batch_tasks", descs, m, tasks.ctypes.data_as(ctypes.c_void_p), n_tasks.value,
               ctypes.byref(n_tasks))
        self.desc = torch.frombuffer(bytearray(bytes(descs)), dtype=torch.uint8).to(device)
        self.tasks = torch.from_numpy(tasks).to(device)
        self.n_matrices, self.n_tasks = m, int(n_tasks.value)
        self.row_off, self.x_off, self.n_groups = row_off, x_off, n_groups
        B = self.s
        B.n_matrices, B.value_type, B.n_tasks = m, _VT[dtype], self.n_tasks
        B.desc, B.tasks = _ptr(self.desc), _ptr(self.tasks)
        B.values, B.columns = _ptr(self.values), _ptr(self.columns)
        B.group_ptr, B.row_lengths = _ptr(self.group_ptr), _ptr(self.row_lengths)
        self.dtype = dtype
        return self

    def spmv(self, x_cat: torch.Tensor, y_cat: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """All members' products; x_cat and y_cat are the concatenated vectors."""
        if x_cat.numel() != self.n_cols_total or x_cat.dtype != self.dtype:
            raise ValueError("x_cat must hold every member's x, in member order")
        y = y_cat if y_cat is not None else torch.empty(self.n_rows_total, dtype=self.dtype, device=x_cat.device)
        L.call("rgcsr_spmv_batched", ctypes.byref(self.s), _ptr(x_cat), _ptr(y), _stream_ptr(stream))
        return y

    def capture(self, x_cat: torch.Tensor, y_cat: torch.Tensor, repeats: int = 1) -> torch.cuda.CUDAGraph:
        """A CUDA graph of `repeats` batched SpMVs on the given buffers."""
        return _capture(self.spmv, x_cat, y_cat, repeats)

    def member_slices(self, i: int):
        return (slice(int(self.x_off[i]), int(self.x_off[i + 1])),
                slice(int(self.row_off[i]), int(self.row_off[i + 1])))


def _capture(spmv, x_cat, y_cat, repeats):
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        spmv(x_cat, y_cat)                             # warm-up outside the capture
        side.synchronize()
        with torch.cuda.graph(g, stream=side):
            for _ in range(repeats):
                spmv(x_cat, y_cat, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    return g


class BlockDiagonalBatch:
    """The batch as one RgCSR matrix diag(A_1, ..., A_m): member i's rows
    follow member i-1's and its column indices are shifted by the column
    counts of the members before it."""

    @classmethod
    def from_csr_list(cls, mats, dtype: torch.dtype = torch.float32, group_size: int = 32,
                      row_order="descending", tile: int | None = 64, variant: int = 0,
                      device="cuda") -> "BlockDiagonalBatch":
        """``mats``: objects with rowptr, col, val, n_rows, n_cols (host
        numpy).  ``row_order`` and ``tile`` as in RgCSRMatrix.from_csr and
        RgCSRMatrix.tile_groups (tile=None: no tile schedule)."""
        from .rgcsr import RgCSRMatrix
        self = cls()
        n_rows = np.array([A.n_rows for A in mats], np.int64)
        n_cols = np.array([A.n_cols for A in mats], np.int64)
        nnz = np.array([A.nnz for A in mats], np.int64)
        self.row_off = np.concatenate([[0], np.cumsum(n_rows)])
        self.x_off = np.concatenate([[0], np.cumsum(n_cols)])
        nnz_off = np.concatenate([[0], np.cumsum(nnz)])
        self.n_rows_total, self.n_cols_total = int(self.row_off[-1]), int(self.x_off[-1])
        if self.n_cols_total > np.iinfo(np.int32).max:
            raise ValueError("the batch has more columns than int32 indices address")
        rowptr = np.concatenate([np.asarray(A.rowptr[:-1], np.int64) + nnz_off[i] for i, A in enumerate(mats)]
                                + [np.array([nnz_off[-1]], np.int64)])
        col = np.concatenate([np.asarray(A.col, np.int64) + self.x_off[i] for i, A in enumerate(mats)]).astype(np.int32)
        npdt = np.float64 if dtype == torch.float64 else np.float32
        val = np.concatenate([np.asarray(A.val).astype(npdt) for A in mats])
        self.M = RgCSRMatrix.from_csr(rowptr, col, val, self.n_cols_total, group_size=group_size, dtype=dtype,
                                      row_order=row_order, device=device)
        del rowptr, col, val
        if tile:
            self.M.tile_groups(tile, variant)
        self.n_matrices, self.nnz, self.dtype = len(mats), int(nnz_off[-1]), dtype
        return self

    def spmv(self, x_cat: torch.Tensor, y_cat: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """All members' products; x_cat and y_cat are the concatenated vectors."""
        return self.M.spmv(x_cat, out=y_cat, stream=stream)

    def capture(self, x_cat: torch.Tensor, y_cat: torch.Tensor, repeats: int = 1) -> torch.cuda.CUDAGraph:
        return _capture(self.spmv, x_cat, y_cat, repeats)

    def member_slices(self, i: int):
        return (slice(int(self.x_off[i]), int(self.x_off[i + 1])),
                slice(int(self.row_off[i]), int(self.row_off[i + 1])))
