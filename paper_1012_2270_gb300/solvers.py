"""Solvers on RgCSR operators (the Krylov setting of the paper's
introduction, where SpMV dominates the cost):

* ``cg``     -- conjugate gradients, one library call (librgcsr's rgcsr_cg).
* ``ir_cg``  -- mixed-precision iterative refinement: FP64 residual and
               update, inner float CG on a lower-precision copy of A
               (rgcsr_ir_cg).
* ``jacobi`` -- damped Jacobi  x_{s+1} = x_s + omega D^{-1} (b - A x_s),
               differentiable with respect to b and the values of A, with
               optional checkpointing (only every k-th iterate is kept;
               segments are recomputed during the backward pass).
"""
from __future__ import annotations

import ctypes

import torch
import torch.utils.checkpoint

from . import _lib as L
from .autograd import SparseOperator
from .rgcsr import RgCSRMatrix, _ptr, _stream_ptr


def _vt(dtype: torch.dtype) -> int:
    return L.F64 if dtype == torch.float64 else L.F32


def cg(A: RgCSRMatrix, b: torch.Tensor, rel_tol: float = 1e-8, max_iter: int = 1000,
       check_every: int = 10):
    """Solves A x = b from x = 0; returns (x, iterations, relative residual)."""
    x = torch.empty_like(b)
    nb = L.lib().rgcsr_cg_workspace_bytes(A.shape[0], A.s.value_type)
    ws = torch.empty(nb, dtype=torch.uint8, device=b.device)
    its, rel = ctypes.c_int32(0), ctypes.c_double(0.0)
    L.call("rgcsr_cg", ctypes.byref(A.s), _ptr(b), _ptr(x), float(rel_tol), int(max_iter), int(check_every),
           _ptr(ws), nb, ctypes.byref(its), ctypes.byref(rel), _stream_ptr())
    return x, its.value, rel.value


def ir_cg(A_hi: RgCSRMatrix, A_lo: RgCSRMatrix, b: torch.Tensor, outer_tol: float = 1e-10,
          max_outer: int = 50, inner_tol: float = 1e-6, max_inner: int = 2000):
    """Iterative refinement; returns (x, corrections, inner iterations, rel. residual)."""
    x = torch.empty_like(b)
    nb = L.lib().rgcsr_ir_cg_workspace_bytes(A_hi.shape[0])
    ws = torch.empty(nb, dtype=torch.uint8, device=b.device)
    outer, inner, rel = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0.0)
    L.call("rgcsr_ir_cg", ctypes.byref(A_hi.s), ctypes.byref(A_lo.s), _ptr(b), _ptr(x), float(outer_tol),
           int(max_outer), float(inner_tol), int(max_inner), _ptr(ws), nb, ctypes.byref(outer),
           ctypes.byref(inner), ctypes.byref(rel), _stream_ptr())
    return x, outer.value, inner.value, rel.value


class _JacobiStep(torch.autograd.Function):
    """One damped-Jacobi step with A's values already loaded in ``op``.

    backward, with lam = dL/dx_{s+1} and w = omega dinv .* lam:
        dL/dx_s = lam - A^T w,   dL/db = w,   dL/da_p = -w[row_p] x_s[col_p].
    """

    @staticmethod
    def forward(ctx, x, b, values, op, dinv, omega):
        n = x.numel()
        Ax = op.A.spmv(x)
        out = torch.empty_like(x)
        L.call("rgcsr_jacobi_step", n, float(omega), _ptr(dinv), _ptr(b), _ptr(Ax), _ptr(x), _ptr(out),
               _vt(x.dtype), _stream_ptr())
        ctx.save_for_backward(x, dinv)
        ctx.op, ctx.omega = op, float(omega)
        return out

    @staticmethod
    def backward(ctx, lam):
        x, dinv = ctx.saved_tensors
        op, omega = ctx.op, ctx.omega
        lam = lam.contiguous()
        n, vt, st = lam.numel(), _vt(lam.dtype), _stream_ptr()
        w = torch.empty_like(lam)
        L.call("rgcsr_diag_scale", n, omega, _ptr(dinv), _ptr(lam), _ptr(w), vt, st)
        dx = db = dval = None
        if ctx.needs_input_grad[0]:
            dx = op.AT.spmv(w)                                     # A^T w
            L.call("rgcsr_axpby", n, 1.0, _ptr(lam), -1.0, _ptr(dx), vt, st)   # lam - A^T w
        if ctx.needs_input_grad[1]:
            db = w
        if ctx.needs_input_grad[2]:
            nw = torch.empty_like(lam)
            L.call("rgcsr_diag_scale", n, -omega, _ptr(dinv), _ptr(lam), _ptr(nw), vt, st)
            dval = op.sampled_dot(nw, x)
        return dx, db, dval, None, None, None


def jacobi(op: SparseOperator, values: torch.Tensor, b: torch.Tensor, dinv: torch.Tensor,
           omega: float, steps: int, checkpoint_every: int = 0) -> torch.Tensor:
    """x_steps of damped Jacobi from x_0 = 0 (dinv fixed, not differentiated).

    checkpoint_every = k > 0 keeps only x_0, x_k, x_2k, ... for the backward
    pass and recomputes each segment of k steps when its gradient is needed."""
    op.set_values(values)

    def segment(x, b, values, k):
        for _ in range(k):
            x = _JacobiStep.apply(x, b, values, op, dinv, omega)
        return x

    x = torch.zeros_like(b)
    if checkpoint_every and checkpoint_every > 0:
        done = 0
        while done < steps:
            k = min(checkpoint_every, steps - done)
            x = torch.utils.checkpoint.checkpoint(segment, x, b, values, k, use_reentrant=False)
            done += k
    else:
        x = segment(x, b, values, steps)
    return x
