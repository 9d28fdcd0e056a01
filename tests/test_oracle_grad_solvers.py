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


# ---------------------------------------------------------------------------
# the error bound of reduced-precision Jacobi gradients (the tolerance of the
# 96^3 FP32 parity test), pinned against an independent float32 evaluation
# ---------------------------------------------------------------------------
def _ell(rowptr, col, val, n):
    """Rows padded to the longest (column 0, value 0): slot j of every row."""
    L = np.diff(rowptr)
    K = int(L.max()) if n else 0
    C = np.zeros((n, K), np.int64)
    V = np.zeros((n, K), np.float64)
    for i in range(n):
        C[i, :L[i]] = col[rowptr[i]:rowptr[i + 1]]
        V[i, :L[i]] = val[rowptr[i]:rowptr[i + 1]]
    return C, V


def _f32_jacobi_grads(A, dinv, b, omega, steps, order):
    """The damped-Jacobi gradient evaluated step by step in float32 (numpy
    rounds every operation to float32): row sums in stored order ("fwd"),
    reversed ("rev"), or each row summed exactly and rounded once ("once",
    like a fused accumulation)."""
    f = np.float32
    n = A.n_rows
    C, V = _ell(A.rowptr, A.col, A.val, n)
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    # A^T in the same padded form
    Ct, Vt = _ell(*_transpose(A.rowptr, A.col, A.val, n), n)
    V32, Vt32 = V.astype(f), Vt.astype(f)

    def matvec(Cm, Vm, Vm32, x):
        if order == "once":
            return (Vm * x.astype(np.float64)[Cm]).sum(axis=1).astype(f)
        js = range(Cm.shape[1]) if order == "fwd" else reversed(range(Cm.shape[1]))
        y = np.zeros(n, f)
        for j in js:
            y = y + Vm32[:, j] * x[Cm[:, j]]
        return y

    d32, b32, w32 = dinv.astype(f), b.astype(f), f(omega)
    xs = [np.zeros(n, f)]
    for _ in range(steps):
        x = xs[-1]
        xs.append(x + (w32 * d32) * (b32 - matvec(C, V, V32, x)))
    lam = f(2) * xs[-1]
    db = np.zeros(n, f)
    dval = np.zeros(A.nnz, f)
    for s in range(steps - 1, -1, -1):
        w = (w32 * d32) * lam
        db = db + w
        dval = dval + ((-w32) * d32 * lam)[rows] * xs[s][A.col]
        lam = lam - matvec(Ct, Vt, Vt32, w)
    return db.astype(np.float64), dval.astype(np.float64)


def _transpose(rowptr, col, val, m):
    trp, tc, perm = oracle.csr_transpose(rowptr, col, m)
    return trp, tc, np.asarray(val)[perm]


def _dominant_matrix(n, seed):
    """Non-symmetric, diagonally dominant, values exact in float32."""
    rng = np.random.default_rng(seed)
    A = synth.random_csr(n, n, rng.integers(2, 9, n), seed=seed)
    A.val = np.round(rng.uniform(-1, 1, A.nnz) * 1024) / 1024
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    off = A.col != rows
    A.val[~off] = 0.0
    dsum = np.bincount(rows[off], np.abs(A.val[off]), minlength=n)
    # make every diagonal entry present: rows without one get it added
    keep = [(i, A.col[A.rowptr[i]:A.rowptr[i + 1]], A.val[A.rowptr[i]:A.rowptr[i + 1]]) for i in range(n)]
    rp, cols, vals = [0], [], []
    for i, c, v in keep:
        c = c.copy(); v = v.copy()
        d = np.ceil((1.0 + dsum[i]) * 8) / 8
        if i in c:
            v[c == i] = d
        else:
            c = np.append(c, i); v = np.append(v, d)
            o = np.argsort(c, kind="stable"); c, v = c[o], v[o]
        cols.append(c); vals.append(v); rp.append(rp[-1] + c.size)
    A.rowptr = np.array(rp, np.int64)
    A.col = np.concatenate(cols).astype(np.int32)
    A.val = np.concatenate(vals)
    return A


@pytest.mark.parametrize("which", ["laplace", "dominant"])
def test_jacobi_grad_bound_holds_for_float32_and_is_not_vacuous(which):
    if which == "laplace":
        A = synth.laplacian_3d(8)
        dinv = np.full(A.n_rows, 1.0 / 6.0)
    else:
        A = _dominant_matrix(300, 4)
        rows = np.repeat(np.arange(A.n_rows), np.diff(A.rowptr))
        dinv = 1.0 / A.val[A.col == rows]
    b = synth.uniform_vector(A.n_rows, seed=2)
    omega, steps = 2.0 / 3.0, 100
    _, db_ref, dval_ref = oracle.jacobi_grad(A.rowptr, A.col, A.val, dinv, b, omega, steps)
    u = 2.0 ** -24
    db_b, dval_b = oracle.jacobi_grad_bound(A.rowptr, A.col, A.val, dinv, b, omega, steps, u)
    worst = 0.0
    for order in ("fwd", "rev", "once"):
        db, dval = _f32_jacobi_grads(A, dinv, b, omega, steps, order)
        e_db, e_dv = np.abs(db - db_ref), np.abs(dval - dval_ref)
        assert (e_db <= db_b).all() and (e_dv <= dval_b).all(), order
        worst = max(worst, (e_db / db_b).max(), (e_dv / dval_b).max())
    # not vacuous: the observed float32 error reaches about 1-3% of it (a
    # worst-case first-order bound against errors that partly cancel), and
    # the same bound for a format with 256x less roundoff is violated
    assert worst > 5e-3
    db_t, dval_t = oracle.jacobi_grad_bound(A.rowptr, A.col, A.val, dinv, b, omega, steps, u / 256)
    db, dval = _f32_jacobi_grads(A, dinv, b, omega, steps, "fwd")
    assert (np.abs(db - db_ref) > db_t).any() or (np.abs(dval - dval_ref) > dval_t).any()
    # and useful: far below the gradients themselves
    assert np.median(dval_b / np.maximum(np.abs(dval_ref), 1e-30)) < 1e-3


def test_jacobi_grad_bound_vanishes_without_rounding_and_grows_with_u():
    A = synth.laplacian_3d(5)
    dinv = np.full(A.n_rows, 1.0 / 6.0)
    b = synth.uniform_vector(A.n_rows, seed=1)
    db0, dv0 = oracle.jacobi_grad_bound(A.rowptr, A.col, A.val, dinv, b, 2 / 3, 20, 0.0)
    assert not db0.any() and not dv0.any()
    db1, dv1 = oracle.jacobi_grad_bound(A.rowptr, A.col, A.val, dinv, b, 2 / 3, 20, 2.0 ** -30)
    db2, dv2 = oracle.jacobi_grad_bound(A.rowptr, A.col, A.val, dinv, b, 2 / 3, 20, 2.0 ** -29)
    # first order in u: doubling u doubles the bound (to within the gamma terms)
    assert np.allclose(db2, 2 * db1, rtol=1e-6) and np.allclose(dv2, 2 * dv1, rtol=1e-6)
