"""Pins for the oracle's Hybrid ELLPACK + COO layout and SpMV (Sec. 3.3) and
for the project's default ELL-width rule (the paper gives none)."""
import numpy as np
import pytest

import oracle
from paper_1012_2270_gb300 import synth


def check_layout(A, K1):
    h = oracle.hyb_layout(A.rowptr, A.col, A.val, K1)
    n = A.n_rows
    L = A.row_lengths()
    # ELL keeps the first min(len, K1) entries of each row, column-major
    for i in range(n):
        for j in range(K1):
            s = j * n + i
            if j < L[i]:
                p = A.rowptr[i] + j
                assert h.ell_col[s] == A.col[p] and h.ell_val[s] == A.val[p]
            else:
                assert h.ell_col[s] == -1 and h.ell_val[s] == 0.0
    # COO holds the rest, in row order then stored order
    exp = [(i, A.col[p], A.val[p]) for i in range(n)
           for p in range(A.rowptr[i] + K1, A.rowptr[i + 1])]
    got = list(zip(h.coo_row.tolist(), h.coo_col.tolist(), h.coo_val.tolist()))
    assert got == [(int(a), int(b), float(c)) for a, b, c in exp]
    assert int((h.ell_col >= 0).sum()) + h.coo_row.size == A.nnz
    return h


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_hyb_layout_and_spmv_every_width(seed):
    rng = np.random.default_rng(seed)
    n, m = 23, 19
    A = synth.random_csr(n, m, rng.integers(0, m + 1, n), seed=seed)
    x = rng.standard_normal(m)
    y_ref, _ = oracle.csr_spmv(A.rowptr, A.col, A.val, x)
    for K1 in range(0, int(A.row_lengths().max()) + 2):
        h = check_layout(A, K1)
        # ELL then COO adds a row's entries in stored order: bit-identical
        assert np.array_equal(oracle.hyb_spmv(h, x), y_ref)


def test_hyb_empty_and_zero_width():
    A = synth.random_csr(5, 4, [0, 0, 0, 0, 0])
    h = oracle.hyb_layout(A.rowptr, A.col, A.val, 0)
    assert h.ell_val.size == 0 and h.coo_row.size == 0
    assert oracle.hyb_spmv(h, np.ones(4)).tolist() == [0.0] * 5


def brute_width(L, sv, si):
    n = len(L)
    best = None
    for K in range(0, max(L) + 1):
        coo = sum(max(0, l - K) for l in L)
        cost = n * K * (sv + si) + 2 * coo * (sv + 2 * si)
        if best is None or cost < best[0]:
            best = (cost, K)
    return best[1]


@pytest.mark.parametrize("sv", [4, 8])
def test_default_width_rule_brute_force(sv):
    rng = np.random.default_rng(sv)
    for _ in range(50):
        n = int(rng.integers(1, 40))
        L = rng.integers(0, 30, n)
        L[rng.integers(0, n)] = rng.integers(0, 200)      # a long row now and then
        A = synth.random_csr(n, 256, L)
        assert oracle.hyb_choose_ell_width(A.rowptr, sv, 4) == brute_width(L.tolist(), sv, 4)


def test_default_width_uniform_rows_is_full_width():
    # interior rows (7 entries) dominate a 20^3 grid: no COO part at all
    A = synth.laplacian_3d(20)
    K = oracle.hyb_choose_ell_width(A.rowptr, 8, 4)
    assert K == 7 and oracle.hyb_coo_count(A.rowptr, K) == 0
    # on a 6^3 grid boundary rows dominate and one slot moves to COO
    A = synth.laplacian_3d(6)
    assert oracle.hyb_choose_ell_width(A.rowptr, 8, 4) == 6
