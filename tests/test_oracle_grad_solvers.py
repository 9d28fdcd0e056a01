"""Pins for the oracle's transposition, SpMM gradients, damped Jacobi with
its adjoint, and conjugate gradients: dense transposes, double transposition,
FP64 central finite differences, dense iteration, and a dense solve."""
import numpy as np
import pytest

import oracle
from paper_1012_2270_gb300 import synth


def dense(rowptr, col, val, n, m):
    D = np.zeros((n, m))
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    D[rows, col] = val
    return D


def test_transpose_dense_and_involution():
    rng = np.random.default_rng(0)
    n, m = 41, 29
    A = synth.random_csr(n, m, rng.integers(0, m + 1, n), seed=0)
    trp, tc, perm = oracle.csr_transpose(A.rowptr, A.col, m)
    D = dense(A.rowptr, A.col, A.val, n, m)
    assert np.array_equal(dense(trp, tc, A.val[perm], m, n), D.T)
    for c in range(m):                       # stable: original rows ascending
        seg = tc[trp[c]:trp[c + 1]]
        assert (np.diff(seg) > 0).all()
    trp2, tc2, perm2 = oracle.csr_transpose(trp, tc, n)
    assert np.array_equal(trp2, A.rowptr) and np.array_equal(tc2, A.col)
    assert np.array_equal(perm[perm2], np.arange(A.nnz))


def test_spmm_grads_dense_and_finite_differences():
    rng = np.random.default_rng(1)
    n, m, k = 13, 11, 3
    A = synth.random_csr(n, m, rng.integers(0, m + 1, n), seed=1)
    X = rng.standard_normal((m, k))
    Y, _ = oracle.csr_spmm(A.rowptr, A.col, A.val, X)
    Gy = 2.0 * Y                                             # loss = ||A X||^2
    dX, dval = oracle.spmm_grads(A.rowptr, A.col, A.val, X, Gy, m)
    D = dense(A.rowptr, A.col, A.val, n, m)
    np.testing.assert_allclose(dX, D.T @ Gy, rtol=1e-12, atol=1e-12)
    rows = np.repeat(np.arange(n), A.row_lengths())
    np.testing.assert_allclose(dval, (Gy @ X.T)[rows, A.col], rtol=1e-12, atol=1e-12)

    def loss(val, X):
        Y, _ = oracle.csr_spmm(A.rowptr, A.col, val, X)
        return float((Y * Y).sum())
    for p in range(A.nnz):
        h = 1e-6 * max(1.0, abs(A.val[p]))
        vp, vm = A.val.copy(), A.val.copy()
        vp[p] += h
        vm[p] -= h
        fd = (loss(vp, X) - loss(vm, X)) / (2 * h)
        assert abs(fd - dval[p]) <= 1e-6 * max(1.0, abs(dval[p]))
    for idx in [(0, 0), (m - 1, k - 1), (m // 2, 1)]:
        h = 1e-6 * max(1.0, abs(X[idx]))
        Xp, Xm = X.copy(), X.copy()
        Xp[idx] += h
        Xm[idx] -= h
        fd = (loss(A.val, Xp) - loss(A.val, Xm)) / (2 * h)
        assert abs(fd - dX[idx]) <= 1e-6 * max(1.0, abs(dX[idx]))


def test_jacobi_forward_matches_dense_iteration():
    A = synth.laplacian_3d(4)
    n = A.n_rows
    b = synth.uniform_vector(n, 0)
    dinv = np.full(n, 1.0 / 6.0)
    x = oracle.jacobi(A.rowptr, A.col, A.val, dinv, b, 2.0 / 3.0, 30)
    D = dense(A.rowptr, A.col, A.val, n, n)
    xr = np.zeros(n)
    for _ in range(30):
        xr = xr + (2.0 / 3.0) * dinv * (b - D @ xr)
    np.testing.assert_allclose(x, xr, rtol=1e-12, atol=1e-13)


def test_jacobi_adjoint_finite_differences():
    A = synth.laplacian_2d(4)
    n = A.n_rows
    rng = np.random.default_rng(3)
    b = rng.uniform(-1, 1, n)
    dinv = np.full(n, 0.25)
    steps, om = 12, 2.0 / 3.0
    loss, db, dval = oracle.jacobi_grad(A.rowptr, A.col, A.val, dinv, b, om, steps)
    xT = oracle.jacobi(A.rowptr, A.col, A.val, dinv, b, om, steps)
    assert loss == pytest.approx(float(xT @ xT), rel=1e-14)

    def f(val, b):
        x = oracle.jacobi(A.rowptr, A.col, val, dinv, b, om, steps)
        return float(x @ x)
    for i in range(n):
        h = 1e-6
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        assert abs((f(A.val, bp) - f(A.val, bm)) / (2 * h) - db[i]) <= 1e-6 * max(1, abs(db[i]))
    for p in range(0, A.nnz, 3):
        h = 1e-6 * max(1.0, abs(A.val[p]))
        vp, vm = A.val.copy(), A.val.copy()
        vp[p] += h
        vm[p] -= h
        assert abs((f(vp, b) - f(vm, b)) / (2 * h) - dval[p]) <= 1e-6 * max(1, abs(dval[p]))


def test_cg_solves_poisson():
    A = synth.laplacian_3d(10)
    n = A.n_rows
    b = synth.uniform_vector(n, 0)
    x, it = oracle.cg(A.rowptr, A.col, A.val, b, 1e-12, 2000)
    D = dense(A.rowptr, A.col, A.val, n, n)
    xr = np.linalg.solve(D, b)
    assert np.linalg.norm(D @ x - b) <= 1e-12 * np.linalg.norm(b) * 1.01
    assert np.linalg.norm(x - xr) <= 1e-10 * np.linalg.norm(xr)
    assert 0 < it < 2000
