"""GPU checks of the solvers built on the SpMV: deterministic dot products,
CG against the oracle's FP64 CG, mixed-precision iterative refinement on the
3D Poisson problem 128^3 (bf16-value inner CG, FP64 outer loop, residual
<= 1e-10), and gradients through 100 damped-Jacobi steps with and without
checkpointing against the oracle's adjoint."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1012_2270_gb300 import synth
from paper_1012_2270_gb300 import _lib as L
from paper_1012_2270_gb300.autograd import SparseOperator
from paper_1012_2270_gb300.rgcsr import RgCSRMatrix, _ptr, _stream_ptr
from paper_1012_2270_gb300 import solvers

pytestmark = pytest.mark.gpu


def gpu_dot(x, y):
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    nb = L.lib().rgcsr_dot_workspace_bytes()
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    vt = L.F64 if x.dtype == torch.float64 else L.F32
    L.call("rgcsr_dot", x.numel(), _ptr(x), _ptr(y), _ptr(out), _ptr(ws), nb, vt, _stream_ptr())
    return float(out)


def test_dot_deterministic_and_exact_on_integers():
    rng = np.random.default_rng(0)
    for n in (0, 1, 1000, 3_000_001):
        a = rng.integers(-50, 51, n).astype(np.float64)
        b = rng.integers(-50, 51, n).astype(np.float64)
        xa, xb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        d1, d2 = gpu_dot(xa, xb), gpu_dot(xa, xb)
        assert d1 == d2 == float(np.dot(a.astype(np.int64), b.astype(np.int64)))
        assert gpu_dot(xa.float(), xb.float()) == d1


def test_float_dot_compensated_accuracy():
    # float vectors: per-thread compensated sums (Dot2) then double.  The
    # second half of the data cancels the first, so the dot product is tiny
    # against sum |x_i y_i|; the result stays within 1e-10 of that sum of the
    # exact dot product of the float inputs (plain float summation: ~1e-7)
    rng = np.random.default_rng(7)
    for n in (1, 777, 2_000_003):
        a = rng.standard_normal(n).astype(np.float32)
        b = rng.standard_normal(n).astype(np.float32)
        h = n // 2
        a[h:2 * h] = a[:h]
        b[h:2 * h] = -b[:h]
        prod = a.astype(np.float64) * b.astype(np.float64)        # exact in double
        exact, scale = float(np.sum(prod)), float(np.sum(np.abs(prod)))
        got = gpu_dot(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
        assert abs(got - exact) <= 1e-10 * scale, (n, got, exact, scale)


@pytest.mark.parametrize("offset", [0, 1])
def test_vector_kernels(offset):
    # offset 0: 16-byte accesses with a tail of n mod W elements; offset 1:
    # vectors that start one element past an aligned address take the
    # scalar path.  FP64 and FP32, n odd.
    rng = np.random.default_rng(1)
    n = 10007

    def dev(v, dt):                         # a CUDA vector starting `offset` elements into its buffer
        buf = torch.zeros(n + 1, dtype=dt, device="cuda")
        t = buf[offset:offset + n]
        t.copy_(torch.from_numpy(v).to(dt))
        return t

    x, y, d, b, ax = (rng.standard_normal(n) for _ in range(5))
    for dt, vt, tol in ((torch.float64, L.F64, 1e-14), (torch.float32, L.F32, 2e-6)):
        xs, ys, ds, bs, axs = (v.astype(np.float64 if dt == torch.float64 else np.float32).astype(np.float64)
                               for v in (x, y, d, b, ax))
        X, Y, D, B, AX = (dev(v, dt) for v in (xs, ys, ds, bs, axs))
        L.call("rgcsr_axpby", n, 2.0, _ptr(X), -0.5, _ptr(Y), vt, _stream_ptr())
        assert np.allclose(Y.double().cpu().numpy(), 2.0 * xs - 0.5 * ys, rtol=tol, atol=tol)
        out = dev(np.zeros(n), dt)
        L.call("rgcsr_jacobi_step", n, 0.7, _ptr(D), _ptr(B), _ptr(AX), _ptr(X), _ptr(out), vt, _stream_ptr())
        assert np.allclose(out.double().cpu().numpy(), xs + 0.7 * ds * (bs - axs), rtol=tol, atol=tol)
        L.call("rgcsr_diag_scale", n, -3.0, _ptr(D), _ptr(X), _ptr(out), vt, _stream_ptr())
        assert np.allclose(out.double().cpu().numpy(), -3.0 * ds * xs, rtol=tol, atol=tol)
        ref = float(np.dot(xs, ds))
        assert abs(gpu_dot(X, D) - ref) <= 1e-12 * float(np.dot(np.abs(xs), np.abs(ds)))
    X = dev(x, torch.float64)
    f = dev(np.zeros(n), torch.float32)
    L.call("rgcsr_convert_vector", n, _ptr(X), L.F64, _ptr(f), L.F32, _stream_ptr())
    assert np.array_equal(f.cpu().numpy(), x.astype(np.float32))
    L.call("rgcsr_convert_vector", n, _ptr(f), L.F32, _ptr(X), L.F64, _stream_ptr())
    assert np.array_equal(X.cpu().numpy(), x.astype(np.float32).astype(np.float64))


def test_stream_read_probe():
    # the bandwidth probe reads and writes nothing; its host checks reject
    # unaligned pointers and sizes before any launch
    from paper_1012_2270_gb300.rgcsr import stream_read
    buf = torch.arange(1 << 20, dtype=torch.float32, device="cuda")
    sink = torch.full((1,), 7.0, device="cuda")
    for nbytes in (0, 16, 4096, 4 << 20):
        L.call("rgcsr_stream_read", _ptr(buf), nbytes, _ptr(sink), _stream_ptr())
    stream_read(buf)
    torch.cuda.synchronize()
    assert float(sink) == 7.0
    assert torch.equal(buf, torch.arange(1 << 20, dtype=torch.float32, device="cuda"))
    lib = L.lib()
    for args in ((_ptr(buf), 20), (ctypes.c_void_p(buf.data_ptr() + 4), 16), (_ptr(buf), -16)):
        assert lib.rgcsr_stream_read(*args, _ptr(sink), _stream_ptr()) == L.RGCSR_ERR_INVALID_ARG


def test_fp64_fma_probe():
    # the FP64 rate probe reports its FMA count and writes nothing
    from paper_1012_2270_gb300.rgcsr import fp64_fma_probe
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert fp64_fma_probe(3) == sms * 2048 * 8 * 3
    sink = torch.full((1,), 5.0, dtype=torch.float64, device="cuda")
    n = ctypes.c_int64(0)
    L.call("rgcsr_fp64_fma_probe", 16, _ptr(sink), ctypes.byref(n), _stream_ptr())
    torch.cuda.synchronize()
    assert float(sink) == 5.0 and n.value == sms * 2048 * 8 * 16
    assert L.lib().rgcsr_fp64_fma_probe(0, _ptr(sink), ctypes.byref(n), _stream_ptr()) == L.RGCSR_ERR_INVALID_ARG


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_cg_against_oracle(dtype):
    A = synth.laplacian_3d(20)
    b = synth.uniform_vector(A.n_rows, seed=0)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, dtype=dtype)
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    x, its, rel = solvers.cg(M, torch.from_numpy(b).to("cuda", dtype), rel_tol=tol, max_iter=2000)
    xr, its_ref = oracle.cg(A.rowptr, A.col, A.val, b, 1e-13, 4000)
    assert rel <= tol and 0 < its < 2000
    xd = x.double().cpu().numpy()
    r, _ = oracle.csr_spmv(A.rowptr, A.col, A.val, xd)
    assert np.linalg.norm(b - r) <= 5 * tol * np.linalg.norm(b)
    assert np.linalg.norm(xd - xr) <= 50 * tol * np.linalg.norm(xr)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_cg_odd_size(dtype):
    # n = 693, not a multiple of a 16-byte pack: the update's scalar tail
    A = synth.laplacian_3d(7, 9, 11)
    b = synth.uniform_vector(A.n_rows, seed=3)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, dtype=dtype)
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    x, its, rel = solvers.cg(M, torch.from_numpy(b).to("cuda", dtype), rel_tol=tol, max_iter=2000)
    assert rel <= tol
    r, _ = oracle.csr_spmv(A.rowptr, A.col, A.val, x.double().cpu().numpy())
    assert np.linalg.norm(b - r) <= 5 * tol * np.linalg.norm(b)


def test_cg_barrier_wait_runs_out():
    # a one-poll limit on the update's grid barriers (64 blocks, so some
    # block polls before the last one arrives): the call reports
    # RGCSR_ERR_TIMEOUT instead of hanging, and the next solve with the
    # default limit is right
    A = synth.laplacian_2d(256)
    b = torch.from_numpy(synth.uniform_vector(A.n_rows, seed=1)).to("cuda", torch.float32)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, dtype=torch.float32)
    assert L.lib().rgcsr_set_wait_limit(1) == L.RGCSR_OK
    try:
        with pytest.raises(L.RgCSRError) as e:
            solvers.cg(M, b, rel_tol=1e-5, max_iter=200)
        assert e.value.status == L.RGCSR_ERR_TIMEOUT
    finally:
        assert L.lib().rgcsr_set_wait_limit(0) == L.RGCSR_OK
    x, its, rel = solvers.cg(M, b, rel_tol=1e-5, max_iter=2000)
    assert rel <= 1e-5
    r, _ = oracle.csr_spmv(A.rowptr, A.col, A.val, x.double().cpu().numpy())
    bn = b.double().cpu().numpy()
    assert np.linalg.norm(bn - r) <= 5e-5 * np.linalg.norm(bn)


def test_cg_zero_rhs():
    A = synth.laplacian_2d(8)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, dtype=torch.float64)
    x, its, rel = solvers.cg(M, torch.zeros(A.n_rows, dtype=torch.float64, device="cuda"))
    assert its == 0 and (x == 0).all()


def ir_solve(A, fmt):
    b = torch.from_numpy(synth.uniform_vector(A.n_rows, seed=0)).cuda()
    M64 = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, dtype=torch.float64)
    lo = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, dtype=torch.float32)
    if fmt != "f32":
        lo = M64.quantized(fmt)
    return (M64, b) + solvers.ir_cg(M64, lo, b, outer_tol=1e-10, max_outer=50, inner_tol=1e-4, max_inner=500)


@pytest.mark.parametrize("fmt", ["bf16", "f16", "f32"])
def test_ir_cg_small_against_oracle(fmt):
    A = synth.laplacian_3d(24)
    M64, b, x, outer, inner, rel = ir_solve(A, fmt)
    assert rel <= 1e-10 and 1 <= outer <= 50
    xr, _ = oracle.cg(A.rowptr, A.col, A.val, b.cpu().numpy(), 1e-13, 5000)
    xd = x.cpu().numpy()
    r, _ = oracle.csr_spmv(A.rowptr, A.col, A.val, xd)
    assert np.linalg.norm(b.cpu().numpy() - r) <= 1.01e-10 * np.linalg.norm(b.cpu().numpy())
    assert np.linalg.norm(xd - xr) <= 1e-8 * np.linalg.norm(xr)


def test_ir_cg_poisson_128():
    A = synth.workload_a()
    M64, b, x, outer, inner, rel = ir_solve(A, "bf16")
    assert rel <= 1e-10
    # certify the residual independently on the host, and compare with an
    # FP64-only CG run on the GPU
    xd = x.cpu().numpy()
    r, _ = oracle.csr_spmv(A.rowptr, A.col, A.val, xd)
    bn = b.cpu().numpy()
    assert np.linalg.norm(bn - r) <= 1.01e-10 * np.linalg.norm(bn)
    x64, its, rel64 = solvers.cg(M64, b, rel_tol=1e-11, max_iter=5000)
    assert np.linalg.norm(xd - x64.cpu().numpy()) <= 1e-8 * np.linalg.norm(x64.cpu().numpy())


def jacobi_problem(nx, dtype, seed=0):
    A = synth.laplacian_3d(nx)
    n = A.n_rows
    b = synth.uniform_vector(n, seed=seed)
    op = SparseOperator(A.rowptr, A.col, A.n_cols, dtype=dtype)
    v = torch.tensor(A.val, dtype=dtype, device="cuda", requires_grad=True)
    bt = torch.tensor(b, dtype=dtype, device="cuda", requires_grad=True)
    dinv = torch.full((n,), 1.0 / 6.0, dtype=dtype, device="cuda")
    return A, b, op, v, bt, dinv


def jacobi_grads(nx, dtype, ck, steps=100):
    A, b, op, v, bt, dinv = jacobi_problem(nx, dtype)
    x = solvers.jacobi(op, v, bt, dinv, 2.0 / 3.0, steps, checkpoint_every=ck)
    loss = (x * x).sum()
    loss.backward()
    return A, b, float(loss.detach()), bt.grad.detach().clone(), v.grad.detach().clone()


def test_jacobi_grads_fp64_against_adjoint():
    A, b, loss, db, dval = jacobi_grads(12, torch.float64, 10)
    loss_ref, db_ref, dval_ref = oracle.jacobi_grad(A.rowptr, A.col, A.val, np.full(A.n_rows, 1 / 6), b,
                                                    2.0 / 3.0, 100)
    assert loss == pytest.approx(loss_ref, rel=1e-12)
    assert np.allclose(db.cpu().numpy(), db_ref, rtol=1e-9, atol=1e-12)
    assert np.allclose(dval.cpu().numpy(), dval_ref, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_checkpointing_is_bit_identical(dtype):
    _, _, l0, db0, dv0 = jacobi_grads(10, dtype, 0)
    _, _, l1, db1, dv1 = jacobi_grads(10, dtype, 10)
    _, _, l2, db2, dv2 = jacobi_grads(10, dtype, 7)
    assert l0 == l1 == l2
    assert torch.equal(db0, db1) and torch.equal(dv0, dv1)
    assert torch.equal(db0, db2) and torch.equal(dv0, dv2)


def test_jacobi_96_checkpointed_fp32_against_adjoint():
    # every element of both gradients within the oracle's float32 error
    # bound (the running-error recursion of the damped-Jacobi adjoint with
    # u = 2^-24, any summation order), not only in norm
    A, b, loss, db, dval = jacobi_grads(96, torch.float32, 10)
    dinv = np.full(A.n_rows, 1 / 6)
    loss_ref, db_ref, dval_ref = oracle.jacobi_grad(A.rowptr, A.col, A.val, dinv, b, 2.0 / 3.0, 100)
    db_b, dval_b = oracle.jacobi_grad_bound(A.rowptr, A.col, A.val, dinv, b, 2.0 / 3.0, 100, 2.0 ** -24)
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    e_db = np.abs(db.double().cpu().numpy() - db_ref)
    e_dv = np.abs(dval.double().cpu().numpy() - dval_ref)
    assert (e_db <= db_b).all(), f"db: worst error/bound {(e_db / db_b).max():.3g}"
    assert (e_dv <= dval_b).all(), f"dval: worst error/bound {(e_dv / dval_b).max():.3g}"
