"""Differentiable sparse products for a fixed sparsity pattern.

``SparseOperator`` keeps, on the GPU, the RgCSR matrix of A, the RgCSR matrix
of A^T (built once from a stable CSR transposition) and the maps from their
slots to the CSR-ordered value array, so values that change between calls
(trainable weights) are refreshed with a gather kernel: into A when a
forward product sees new values, into A^T when a backward product needs
them; values the matrix already holds (same content, checked on the
device by a hash) are not gathered again.

``spmm(op, values, X)`` computes A X (X a vector or an [n_cols, k] block) and
is differentiable with respect to both the values and X:
    dX      = A^T dY                      (RgCSR SpMV/SpMM of A^T)
    dA_p    = sum_b dY[row_p, b] X[col_p, b]   (sampled dot over the pattern)
Every product and gradient runs in librgcsr's kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L
from .rgcsr import RgCSRMatrix, _dev, _ptr, _stream_ptr, csr_struct


class SparseOperator:
    """A fixed CSR pattern (``rowptr``, ``col``) of shape [n_rows, n_cols]."""

    def __init__(self, rowptr, col, n_cols: int, dtype: torch.dtype = torch.float32,
                 group_size: int = 32, long_rows: tuple | None = None, row_order=None,
                 tiles: int | None = None, device="cuda"):
        """For uneven rows, A and A^T can take a launch schedule: long_rows =
        (threshold, segment) for the long-row segments (lanes-per-row SpMM),
        or row_order="descending" with tiles = C for group tiles of C
        slot-rows (tiled SpMV/SpMM, group_size <= 32)."""
        self.rowptr = _dev(rowptr, torch.int64, device)
        self.col = _dev(col, torch.int32, device)
        self.n_rows = self.rowptr.numel() - 1
        self.n_cols = int(n_cols)
        self.nnz = self.col.numel()
        self.dtype = dtype
        zeros = torch.zeros(self.nnz, dtype=dtype, device=device)
        st = _stream_ptr()
        self.A = RgCSRMatrix.from_csr(self.rowptr, self.col, zeros, self.n_cols, group_size=group_size,
                                      dtype=dtype, keep_slot_map=True, row_order=row_order)
        # stable transposition of the pattern
        csr = csr_struct(self.rowptr, self.col, zeros, self.n_cols)
        nb = L.lib().rgcsr_transpose_workspace_bytes(self.nnz, self.n_rows, self.n_cols)
        ws = torch.empty(nb, dtype=torch.uint8, device=device)
        t_rowptr = torch.empty(self.n_cols + 1, dtype=torch.int64, device=device)
        t_col = torch.empty(self.nnz, dtype=torch.int32, device=device)
        perm = torch.empty(self.nnz, dtype=torch.int64, device=device)
        L.call("rgcsr_csr_transpose", ctypes.byref(csr), _ptr(t_rowptr), _ptr(t_col), _ptr(perm),
               None, _ptr(ws), nb, st)
        del ws
        self.AT = RgCSRMatrix.from_csr(t_rowptr, t_col, zeros, self.n_rows, group_size=group_size,
                                       dtype=dtype, keep_slot_map=True, row_order=row_order)
        self.at_src = torch.empty(self.AT.n_stored, dtype=torch.int64, device=device)
        L.call("rgcsr_compose_index", _ptr(self.AT.slot_to_csr), _ptr(perm), self.AT.n_stored,
               _ptr(self.at_src), st)
        # what values A and A^T hold (device records: zero = nothing yet)
        self._a_state = torch.zeros(L.VALUES_STATE_BYTES // 8, dtype=torch.int64, device=device)
        self._at_state = torch.zeros(L.VALUES_STATE_BYTES // 8, dtype=torch.int64, device=device)
        self.row_index = torch.empty(self.nnz, dtype=torch.int32, device=device)
        L.call("rgcsr_csr_row_index", ctypes.byref(csr), _ptr(self.row_index), st)
        if long_rows is not None:
            self.A.split_long_rows(*long_rows)
            self.AT.split_long_rows(*long_rows)
        if tiles is not None:
            self.A.tile_groups(tiles)
            self.AT.tile_groups(tiles)

    def load_values(self, values: torch.Tensor, transposed: bool = False, force: bool = False) -> None:
        """Loads CSR-ordered values into the RgCSR matrix of A (or of A^T)
        unless that matrix already holds them: the library hashes the values
        on the device and gathers only when the hash differs from the one it
        recorded for the matrix (rgcsr_gather_values_if_changed), so a
        change made any way -- in place, through ``.data``, by another
        kernel -- is seen, and unchanged values cost one read instead of a
        gather.  force=True forgets the record first."""
        if values.dtype != self.dtype or values.numel() != self.nnz or not values.is_contiguous():
            raise ValueError(f"values must be a contiguous {self.dtype} vector of length {self.nnz}")
        M, src, state = (self.AT, self.at_src, self._at_state) if transposed else \
            (self.A, self.A.slot_to_csr, self._a_state)
        if force:
            state.zero_()
        L.call("rgcsr_gather_values_if_changed", ctypes.byref(M.s), _ptr(values), self.nnz, _ptr(src),
               _ptr(state), _stream_ptr())

    def set_values(self, values: torch.Tensor, force: bool = False) -> None:
        """Loads CSR-ordered values into the RgCSR matrices of A and A^T."""
        self.load_values(values, False, force)
        self.load_values(values, True, force)

    def matmul(self, X: torch.Tensor) -> torch.Tensor:
        return self.A.spmv(X) if X.dim() == 1 else self.A.spmm(X)

    def matmul_t(self, G: torch.Tensor) -> torch.Tensor:
        return self.AT.spmv(G) if G.dim() == 1 else self.AT.spmm(G)

    def sampled_dot(self, G: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
        """out[p] = sum_b G[row_p, b] X[col_p, b] for every stored entry p."""
        G2 = G.reshape(self.n_rows, -1)
        X2 = X.reshape(self.n_cols, -1)
        k = G2.shape[1]
        if X2.shape[1] != k or G2.stride(1) != 1 or X2.stride(1) != 1:
            raise ValueError("G and X need the same number of columns and unit column stride")
        out = torch.empty(self.nnz, dtype=self.dtype, device=G.device)
        vt = L.F64 if self.dtype == torch.float64 else L.F32
        L.call("rgcsr_sampled_dot", self.nnz, k, _ptr(self.row_index), _ptr(self.col), _ptr(G2),
               max(G2.stride(0), k), _ptr(X2), max(X2.stride(0), k), _ptr(out), vt, _stream_ptr())
        return out


class _SparseMatmul(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, X, op):
        op.load_values(values)                 # A only; A^T is loaded by the backward that needs it
        ctx.op = op
        ctx.save_for_backward(values, X)
        return op.matmul(X.contiguous())

    @staticmethod
    def backward(ctx, dY):
        values, X = ctx.saved_tensors
        op = ctx.op
        dY = dY.contiguous()
        d_values = op.sampled_dot(dY, X.contiguous()) if ctx.needs_input_grad[0] else None
        dX = None
        if ctx.needs_input_grad[1]:
            op.load_values(values, transposed=True)    # skipped if A^T already holds them
            dX = op.matmul_t(dY)
        return d_values, dX, None


def spmm(op: SparseOperator, values: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
    """A X with A = (op's pattern, values); differentiable in values and X."""
    return _SparseMatmul.apply(values, X, op)
