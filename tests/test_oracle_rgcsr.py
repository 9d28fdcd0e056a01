"""Pins for the oracle's RgCSR layout builder and SpMV semantics (Sec. 3.4):
the paper's worked-example counts, brute force over every small row-length
pattern with an independently written address map, the padding/NaN
behaviour that separates RgCSR from sliced ELLPACK, and the optimality of
descending ordering (Sec. 4.4.2)."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_1012_2270_gb300 import synth


def csr_from_lengths(L, m=None, seed=0):
    L = np.asarray(L, dtype=np.int64)
    m = m or max(int(L.max(initial=0)), 1)
    return synth.random_csr(L.size, m, L, seed=seed)


def test_worked_example(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "worked_example.json")))
    L = np.array(g["row_lengths"])
    # the row lengths follow from the first-entry positions and nnz
    starts = g["first_entry_positions"] + [g["nnz"]]
    assert np.diff(starts).tolist() == L.tolist()
    A = csr_from_lengths(L, m=8)
    lay = oracle.rgcsr_layout(A.rowptr, A.col, A.val, g["group_size"])
    assert lay.group_ptr.tolist() == g["rgcsr_group_ptr"]
    assert lay.n_stored - A.nnz == g["rgcsr_artificial_zeros"]
    assert int((lay.slot_to_csr < 0).sum()) == g["rgcsr_artificial_zeros"]
    h = oracle.hyb_layout(A.rowptr, A.col, A.val, g["ellpack_width"])
    assert h.coo_row.size == 0
    assert int((h.ell_col < 0).sum()) == g["ellpack_artificial_zeros"]


def independent_map(L, G):
    """Address of (row, slot) written out from the format description."""
    n = len(L)
    addr = {}
    off = 0
    for g0 in range(0, n, G):
        rows = list(range(g0, min(g0 + G, n)))
        K = max(L[i] for i in rows)
        for j in range(K):
            for t, i in enumerate(rows):
                addr[(i, j)] = off + j * len(rows) + t
        off += K * len(rows)
    return addr, off


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_brute_force_all_length_patterns(n):
    for G in (1, 2, 4):
        for L in itertools.product(range(5), repeat=n):
            A = csr_from_lengths(L, m=5, seed=sum(L))
            lay = oracle.rgcsr_layout(A.rowptr, A.col, A.val, G)
            addr, total = independent_map(L, G)
            assert lay.n_stored == total
            assert lay.row_lengths.tolist() == list(L)
            # rowLengths and groupPointers alone: group g starts where the
            # address map puts slot 0 of its first row, or, for a group of
            # empty rows, where the previous group ends
            rl, gp = oracle.rgcsr_sizes(A.rowptr, G)
            assert rl.tolist() == list(L)
            starts = [addr.get((g0, 0)) for g0 in range(0, n, G)]
            for g in range(len(starts) - 1, -1, -1):
                if starts[g] is None:
                    starts[g] = starts[g + 1] if g + 1 < len(starts) else total
            assert gp.tolist() == starts + [total]
            assert np.array_equal(gp, lay.group_ptr)
            seen = np.zeros(lay.n_stored, bool)
            for i in range(n):
                for j in range(L[i]):
                    s = addr[(i, j)]
                    p = A.rowptr[i] + j
                    assert lay.slot_to_csr[s] == p
                    assert lay.columns[s] == A.col[p]
                    assert lay.values[s] == A.val[p]
                    seen[s] = True
            pad = ~seen
            assert (lay.slot_to_csr[pad] == -1).all()
            assert (lay.columns[pad] == 0).all()
            assert (lay.values[pad].view(np.uint64) == 0).all()
            x = np.arange(1.0, 6.0) * 0.37
            y_ref, _ = oracle.csr_spmv(A.rowptr, A.col, A.val, x)
            assert np.array_equal(oracle.rgcsr_spmv(lay, x), y_ref)


@pytest.mark.parametrize("G", [1, 3, 8, 32, 33, 128])
def test_rgcsr_spmv_dense_and_ragged_tail(G):
    rng = np.random.default_rng(G)
    n, m = 301, 97          # n not a multiple of G: a partial last group
    A = synth.random_csr(n, m, rng.integers(0, 20, n), seed=G)
    x = rng.standard_normal(m)
    lay = oracle.rgcsr_layout(A.rowptr, A.col, A.val, G)
    D = np.zeros((n, m))
    rows = np.repeat(np.arange(n), A.row_lengths())
    D[rows, A.col] = A.val
    np.testing.assert_allclose(oracle.rgcsr_spmv(lay, x), D @ x, rtol=1e-13, atol=1e-13)
    # padding count: sum over groups of R_g * K_g minus nnz
    L = A.row_lengths()
    total = sum(len(L[g:g + G]) * L[g:g + G].max() for g in range(0, n, G))
    assert lay.n_stored == total


def test_padding_is_never_multiplied():
    # rows 0..3 never touch column 0; x[0] = NaN.  RgCSR stays finite; the
    # sliced-ELLPACK reading of the same slabs multiplies the padding (whose
    # ghost column is 0) and turns the short rows into NaN.
    L = [1, 3, 2, 3]
    A = csr_from_lengths(L, m=6, seed=3)
    A.col = A.col.copy()
    A.col[:] = np.concatenate([np.sort(np.random.default_rng(i).choice(np.arange(1, 6), l, replace=False))
                               for i, l in enumerate(L)]).astype(np.int32)
    lay = oracle.rgcsr_layout(A.rowptr, A.col, A.val, 4)
    x = np.ones(6)
    x[0] = np.nan
    y = oracle.rgcsr_spmv(lay, x)
    assert np.isfinite(y).all()
    ys = oracle.sliced_ell_spmv(lay, x)
    short = np.array(L) < max(L)
    assert np.isnan(ys[short]).all() and np.isfinite(ys[~short]).all()
    x[0] = 1.0          # with a finite ghost target both readings agree
    np.testing.assert_allclose(oracle.sliced_ell_spmv(lay, x), y, rtol=1e-15)


def test_zero_padding_iff_equal_lengths_per_group():
    rng = np.random.default_rng(9)
    for _ in range(200):
        G = int(rng.integers(1, 6))
        L = rng.integers(0, 4, int(rng.integers(1, 12)))
        A = csr_from_lengths(L, m=4)
        lay = oracle.rgcsr_layout(A.rowptr, A.col, A.val, G)
        equal = all(len(set(L[g:g + G].tolist())) == 1 for g in range(0, L.size, G))
        assert (lay.n_stored == A.nnz) == equal
        if A.nnz:
            assert oracle.artificial_zero_percent(A.nnz, lay.n_stored) >= 0.0


def test_artificial_zero_percent_definition():
    # 100% = as many artificial zeros as non-zeros (Sec. 4.3)
    assert oracle.artificial_zero_percent(10, 20) == 100.0
    assert oracle.artificial_zero_percent(13, 20) == pytest.approx(700 / 13)


@pytest.mark.parametrize("n,G", [(4, 2), (4, 4), (6, 2), (6, 3), (8, 4)])
def test_descending_order_minimises_padding(n, G):
    # Sec. 4.4.2 calls descending ordering optimal for suppressing artificial
    # zeros; that holds when every group is full (G divides n).
    rng = np.random.default_rng(n * 10 + G)
    perms = list(itertools.permutations(range(n))) if n <= 6 else None
    for _ in range(10):
        L = rng.integers(0, 6, n)
        A = csr_from_lengths(L, m=6)
        perm = oracle.descending_order(A.rowptr)
        assert sorted(perm.tolist()) == list(range(n))
        Lp = L[perm]
        assert (np.diff(Lp) <= 0).all()
        if perms is not None:
            best = min(independent_map([L[p] for p in q], G)[1] for q in perms)
        else:  # full groups: any order with sorted contiguous groups is optimal
            best = independent_map(sorted(L.tolist()), G)[1]
        assert independent_map(Lp.tolist(), G)[1] == best
        for a, b in zip(perm[:-1], perm[1:]):       # stable on ties
            if L[a] == L[b]:
                assert a < b


def test_descending_not_optimal_with_partial_last_group():
    # With a partial last group the longest rows are better placed there:
    # lengths [5,1,1,1], G = 3 -> descending stores 3*5 + 1 = 16 slots,
    # the order [1,1,1,5] stores 3*1 + 5 = 8.
    assert independent_map([5, 1, 1, 1], 3)[1] == 16
    assert independent_map([1, 1, 1, 5], 3)[1] == 8


def test_full_size_counts_stencil():
    A = synth.laplacian_3d(32)
    lay = oracle.rgcsr_layout(A.rowptr, A.col, A.val, 32)
    # 32 consecutive rows are one x-line of the grid: padding only where a
    # line mixes boundary and interior rows
    assert lay.n_stored >= A.nnz
    x = synth.uniform_vector(A.n_cols, 0)
    y, _ = oracle.csr_spmv(A.rowptr, A.col, A.val, x)
    assert np.array_equal(oracle.rgcsr_spmv(lay, x), y)


def dense_of(rowptr, col, val, n_cols):
    D = np.zeros((len(rowptr) - 1, n_cols))
    for i in range(len(rowptr) - 1):
        for p in range(rowptr[i], rowptr[i + 1]):
            D[i, col[p]] += float(val[p])
    return D


@pytest.mark.parametrize("seed", range(6))
def test_permute_rows_is_row_permutation_of_dense(seed):
    # Row ordering (Sec. 4.4.2, Table 7) stores P A: row k of the reordered
    # matrix is row perm[k] of A, entry for entry
    rng = np.random.default_rng(seed)
    n, m = 9, 7
    A = csr_from_lengths(rng.integers(0, 6, n), m=m, seed=seed)
    perm = rng.permutation(n)
    rp, c, v, src = oracle.permute_rows(A.rowptr, A.col, A.val, perm)
    assert np.array_equal(dense_of(rp, c, v, m), dense_of(A.rowptr, A.col, A.val, m)[perm])
    assert np.array_equal(A.col[src], c) and np.array_equal(A.val[src], v)
    assert sorted(src.tolist()) == list(range(A.nnz))
    with pytest.raises(ValueError):
        oracle.permute_rows(A.rowptr, A.col, A.val, np.zeros(n, np.int64))


@pytest.mark.parametrize("G", [1, 2, 3, 4])
def test_reordered_layout(G):
    rng = np.random.default_rng(G)
    n, m = 11, 8
    L = rng.integers(0, 7, n)
    A = csr_from_lengths(L, m=m, seed=G)
    x = rng.uniform(-1, 1, m)
    plain = oracle.rgcsr_layout(A.rowptr, A.col, A.val, G)
    same = oracle.rgcsr_layout(A.rowptr, A.col, A.val, G, row_order=np.arange(n))
    for f in ("row_lengths", "group_ptr", "values", "columns", "slot_to_csr"):
        assert np.array_equal(getattr(plain, f), getattr(same, f)), f
    perm = oracle.descending_order(A.rowptr)
    lay = oracle.rgcsr_layout(A.rowptr, A.col, A.val, G, row_order=perm)
    # the address map of the format applied to the reordered lengths
    addr, total = independent_map(L[perm].tolist(), G)
    assert lay.n_stored == total
    assert lay.row_lengths.tolist() == L[perm].tolist()
    for k in range(n):
        i = perm[k]
        for j in range(L[i]):
            a = addr[(k, j)]
            assert lay.slot_to_csr[a] == A.rowptr[i] + j
            assert lay.values[a] == A.val[A.rowptr[i] + j] and lay.columns[a] == A.col[A.rowptr[i] + j]
    pad = lay.slot_to_csr < 0
    assert (lay.values[pad] == 0).all() and (lay.columns[pad] == 0).all()
    # y comes back in A's row order: the same sums as the plain CSR product
    y, _ = oracle.csr_spmv(A.rowptr, A.col, A.val, x)
    assert np.array_equal(oracle.rgcsr_spmv(lay, x), y)
    assert np.allclose(y, dense_of(A.rowptr, A.col, A.val, m) @ x, rtol=0, atol=1e-12)
