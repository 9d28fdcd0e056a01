"""Pins for the oracle's CSR SpMV / SpMM (Sec. 3.1) against definitions that
do not go through it: dense products, identity, diagonal and permutation
matrices, row sums, and the |A||x| error scale."""
import math

import numpy as np
import pytest

import oracle
from paper_1012_2270_gb300 import synth


def dense(A):
    D = np.zeros((A.n_rows, A.n_cols))
    rows = np.repeat(np.arange(A.n_rows), A.row_lengths())
    np.add.at(D, (rows, A.col), A.val)
    return D


@pytest.mark.parametrize("n,m,seed", [(1, 1, 0), (7, 5, 1), (33, 64, 2), (64, 17, 3)])
def test_csr_spmv_matches_dense(n, m, seed):
    rng = np.random.default_rng(seed)
    L = rng.integers(0, m + 1, n)
    A = synth.random_csr(n, m, L, seed=seed)
    x = rng.standard_normal(m)
    y, ay = oracle.csr_spmv(A.rowptr, A.col, A.val, x)
    D = dense(A)
    np.testing.assert_allclose(y, D @ x, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(ay, np.abs(D) @ np.abs(x), rtol=1e-13, atol=1e-13)


def test_nonsymmetric_catches_transpose():
    # A deliberately non-symmetric 2x3 case: y = [1*x0 + 2*x2, 3*x1]
    rowptr = np.array([0, 2, 3])
    col = np.array([0, 2, 1])
    val = np.array([1.0, 2.0, 3.0])
    y, _ = oracle.csr_spmv(rowptr, col, val, np.array([10.0, 100.0, 1000.0]))
    assert y.tolist() == [2010.0, 300.0]


def test_identity_diagonal_permutation_exact():
    n = 50
    rng = np.random.default_rng(0)
    x = rng.standard_normal(n)
    I_rp = np.arange(n + 1)
    I_c = np.arange(n)
    y, _ = oracle.csr_spmv(I_rp, I_c, np.ones(n), x)
    assert np.array_equal(y, x)
    d = rng.standard_normal(n)
    y, _ = oracle.csr_spmv(I_rp, I_c, d, x)
    assert np.array_equal(y, d * x)
    perm = rng.permutation(n)
    y, _ = oracle.csr_spmv(I_rp, perm, np.ones(n), x)
    assert np.array_equal(y, x[perm])


def test_row_sums_exact_on_integers():
    # A.1 = row sums; small integer values make every partial sum exact.
    rng = np.random.default_rng(5)
    A = synth.random_csr(40, 30, rng.integers(0, 31, 40), seed=5)
    A.val = rng.integers(-8, 9, A.nnz).astype(np.float64)
    y, _ = oracle.csr_spmv(A.rowptr, A.col, A.val, np.ones(A.n_cols))
    sums = [math.fsum(A.val[A.rowptr[i]:A.rowptr[i + 1]]) for i in range(A.n_rows)]
    assert y.tolist() == sums


def test_empty_rows_and_empty_matrix():
    y, ay = oracle.csr_spmv(np.zeros(4, np.int64), np.zeros(0), np.zeros(0), np.ones(3))
    assert y.tolist() == [0.0, 0.0, 0.0] and ay.tolist() == [0.0, 0.0, 0.0]
    y, _ = oracle.csr_spmv(np.zeros(1, np.int64), np.zeros(0), np.zeros(0), np.ones(0))
    assert y.size == 0


def test_laplacian_counts_and_values():
    A = synth.workload_small_laplacian()
    assert (A.n_rows, A.nnz) == (4096, 20224)
    # interior rows of the Laplacian annihilate constants; all rows sum to
    # 4 - (number of neighbours)
    y, _ = oracle.csr_spmv(A.rowptr, A.col, A.val, np.ones(A.n_cols))
    assert y.min() == 0.0 and y.max() == 2.0
    assert synth.laplacian_3d(8).nnz == 7 * 512 - 6 * 64


@pytest.mark.parametrize("k", [1, 4, 8])
def test_csr_spmm_matches_dense(k):
    rng = np.random.default_rng(k)
    A = synth.random_csr(37, 23, rng.integers(0, 24, 37), seed=k)
    X = rng.standard_normal((23, k))
    Y, aY = oracle.csr_spmm(A.rowptr, A.col, A.val, X)
    D = dense(A)
    np.testing.assert_allclose(Y, D @ X, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(aY, np.abs(D) @ np.abs(X), rtol=1e-13, atol=1e-13)
    # each column of the SpMM is the SpMV of that column
    for b in range(k):
        y, _ = oracle.csr_spmv(A.rowptr, A.col, A.val, X[:, b])
        assert np.array_equal(Y[:, b], y)


def test_peak_model_table(golden_dir):
    import json, os
    g = json.load(open(os.path.join(golden_dir, "peak_table.json")))
    for c in g["cases"]:
        got = oracle.peak_gflops(g["bandwidth_gbs"], c["value_bytes"], g["index_bytes"], c["x_cached"])
        assert round(got, 2) == c["gflops"], c
