"""GPU parity of the multi-RHS product Y = A X against the oracle's CSR
SpMM, elementwise within tau*(|A||X|): column counts that exercise every
chunk width and ragged remainders, strided X and Y, long rows, reduced
precision storage, and matrix (b) at k = 1, 4, 8, 16, 32."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TAU, assert_within_bound, rounded_values
from paper_1012_2270_gb300 import synth
from paper_1012_2270_gb300.rgcsr import RgCSRMatrix

pytestmark = pytest.mark.gpu

NP = {"f32": np.float32, "f64": np.float64}
TT = {"f32": torch.float32, "f64": torch.float64}


def check(A, M, dtype, X, tau, vals=None, X_dev=None, Y_out=None):
    Xd = X_dev if X_dev is not None else torch.from_numpy(X.astype(NP[dtype])).cuda()
    Y = M.spmm(Xd, out=Y_out).cpu().numpy()
    v = rounded_values(A.val, dtype) if vals is None else vals
    Y_ref, aY = oracle.csr_spmm(A.rowptr, A.col, v, X.astype(NP[dtype]).astype(np.float64))
    assert_within_bound(Y.ravel(), Y_ref.ravel(), aY.ravel(), tau, f"{A.name} {dtype} k={X.shape[1]}")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8, 16, 17, 32, 33, 40])
def test_spmm_ragged(dtype, k):
    rng = np.random.default_rng(k)
    Ls = rng.integers(0, 30, 1500)
    Ls[[3, 700, 701]] = [2000, 900, 35]
    A = synth.random_csr(1500, 2500, Ls, seed=k)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, dtype=TT[dtype])
    X = synth.uniform_matrix(A.n_cols, k, seed=k)
    check(A, M, dtype, X, TAU[dtype])


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_spmm_strided_operands_and_group_sizes(dtype):
    rng = np.random.default_rng(9)
    A = synth.random_csr(777, 500, rng.integers(0, 20, 777), seed=9)
    for G in (1, 16, 32, 64):
        M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=G,
                                 dtype=TT[dtype])
        wide = synth.uniform_matrix(A.n_cols, 11, seed=G)
        X = wide[:, 2:9]                                     # k = 7, row stride 11
        Xd = torch.from_numpy(wide.astype(NP[dtype])).cuda()[:, 2:9]
        Yw = torch.full((A.n_rows, 10), 7.0, dtype=TT[dtype], device="cuda")
        check(A, M, dtype, X, TAU[dtype], X_dev=Xd, Y_out=Yw[:, 1:8])
        assert (Yw[:, 0] == 7.0).all() and (Yw[:, 8:] == 7.0).all()   # untouched


def test_spmm_matches_spmv_columns():
    A = synth.workload_small_laplacian()
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, dtype=torch.float64)
    X = torch.from_numpy(synth.uniform_matrix(A.n_cols, 4, seed=0)).cuda()
    Y = M.spmm(X)
    for b in range(4):
        y = M.spmv(X[:, b].contiguous())
        assert torch.allclose(Y[:, b], y, rtol=0, atol=1e-12)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_spmm_quantized(fmt):
    rng = np.random.default_rng(5)
    A = synth.random_csr(900, 600, rng.integers(0, 25, 900), seed=5)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, dtype=torch.float64)
    Q = M.quantized(fmt)
    q, s = oracle.quantize_rows(A.rowptr, A.val, oracle.BF16 if fmt == "bf16" else oracle.F16)
    deq = oracle.dequantized_values(A.rowptr, q, s, oracle.BF16 if fmt == "bf16" else oracle.F16)
    X = synth.uniform_matrix(A.n_cols, 8, seed=1)
    check(A, Q, "f32", X, 2e-6, vals=deq)


@pytest.mark.parametrize("k", [1, 4, 8, 16, 32])
def test_spmm_full_size_b(k):
    A = synth.workload_b()
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(np.float32), A.n_cols, dtype=torch.float32)
    X = synth.uniform_matrix(A.n_cols, k, seed=k)
    check(A, M, "f32", X, TAU["f32"])


# ---------------------------------------------------------------------------
# lanes-per-row kernels (rgcsr_spmm_long_rows), with and without the
# long-row segment schedule
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("k", [1, 3, 4, 5, 8, 16, 17, 32, 33, 40])
@pytest.mark.parametrize("G,sched", [(1, (16, 64)), (32, (0, 7)), (3, None)])
def test_spmm_rows_ragged(dtype, k, G, sched):
    rng = np.random.default_rng(k + G)
    Ls = rng.integers(0, 30, 1500)
    Ls[[3, 700, 701]] = [2000, 900, 35]
    A = synth.random_csr(1500, 2500, Ls, seed=k)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=G, dtype=TT[dtype])
    if sched:
        M.split_long_rows(*sched)
    Xd = torch.from_numpy(synth.uniform_matrix(A.n_cols, k, seed=k).astype(NP[dtype])).cuda()
    Y = M.spmm(Xd, rows=True).cpu().numpy()
    Y_ref, aY = oracle.csr_spmm(A.rowptr, A.col, rounded_values(A.val, dtype), Xd.cpu().numpy().astype(np.float64))
    assert_within_bound(Y.ravel(), Y_ref.ravel(), aY.ravel(), TAU[dtype], f"rows k={k} G={G} {sched}")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_spmm_rows_strided_and_reordered(dtype):
    rng = np.random.default_rng(4)
    A = synth.random_csr(901, 700, rng.integers(0, 40, 901), seed=4)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=32,
                             dtype=TT[dtype], row_order="descending").split_long_rows(8, 16)
    wide = synth.uniform_matrix(A.n_cols, 19, seed=2)
    Xd = torch.from_numpy(wide.astype(NP[dtype])).cuda()[:, 3:16]        # k = 13, unaligned rows
    Yw = torch.full((A.n_rows, 15), 5.0, dtype=TT[dtype], device="cuda")
    M.spmm(Xd, out=Yw[:, 1:14])
    assert (Yw[:, 0] == 5.0).all() and (Yw[:, 14] == 5.0).all()
    Y_ref, aY = oracle.csr_spmm(A.rowptr, A.col, rounded_values(A.val, dtype), wide[:, 3:16].astype(NP[dtype]).astype(np.float64))
    assert_within_bound(Yw[:, 1:14].cpu().numpy().ravel(), Y_ref.ravel(), aY.ravel(), TAU[dtype], "rows strided")


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_spmm_rows_quantized(fmt):
    A = synth.power_law(20_000, seed=8)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=1, dtype=torch.float64)
    Q = M.quantized(fmt).split_long_rows(32, 128)
    code = oracle.BF16 if fmt == "bf16" else oracle.F16
    q, s = oracle.quantize_rows(A.rowptr, A.val, code)
    deq = oracle.dequantized_values(A.rowptr, q, s, code)
    X = synth.uniform_matrix(A.n_cols, 12, seed=3)
    Y = Q.spmm(torch.from_numpy(X.astype(np.float32)).cuda()).cpu().numpy()
    Y_ref, aY = oracle.csr_spmm(A.rowptr, A.col, deq, X.astype(np.float32).astype(np.float64))
    assert_within_bound(Y.ravel(), Y_ref.ravel(), aY.ravel(), 2e-6, f"rows {fmt}")


def test_spmm_rows_partials_too_small():
    import ctypes
    from paper_1012_2270_gb300 import _lib as L
    from paper_1012_2270_gb300.rgcsr import _ptr, _stream_ptr
    A = synth.power_law(5000, seed=1)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(np.float32), A.n_cols, group_size=1,
                             dtype=torch.float32).split_long_rows(16, 64)
    assert M.n_long_segments > 0
    X = torch.zeros(A.n_cols, 8, device="cuda")
    Y = torch.empty(A.n_rows, 8, device="cuda")
    part = torch.empty(M.n_long_segments * 8 - 1, device="cuda")
    st = L.lib().rgcsr_spmm_long_rows(ctypes.byref(M.s), ctypes.byref(M._long[0]), 8, _ptr(X), 8, _ptr(Y), 8,
                                      _ptr(part), part.numel(), _stream_ptr())
    assert st == L.RGCSR_ERR_WORKSPACE


@pytest.mark.parametrize("k,sched", [(4, (32, 256)), (16, (16, 64)), (32, (16, 64))])
def test_spmm_rows_full_size_b(k, sched):
    # (16, 64): the schedule the benchmark's SpMM form times
    A = synth.workload_b()
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(np.float32), A.n_cols, group_size=1,
                             dtype=torch.float32).split_long_rows(*sched)
    X = synth.uniform_matrix(A.n_cols, k, seed=k)
    check(A, M, "f32", X, TAU["f32"])


# ---------------------------------------------------------------------------
# tiled kernels (rgcsr_spmm_tiles) on the group-tile schedule
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("k", [1, 2, 4, 5, 8, 13, 32])
@pytest.mark.parametrize("G,order,C", [(32, "descending", 16), (32, None, 1 << 20), (7, None, 3)])
def test_spmm_tiles_ragged(dtype, k, G, order, C):
    rng = np.random.default_rng(k * 3 + G)
    Ls = rng.integers(0, 30, 1500)
    Ls[[3, 700, 701]] = [2000, 900, 35]
    A = synth.random_csr(1500, 2500, Ls, seed=k + 1)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=G, dtype=TT[dtype],
                             row_order=order).tile_groups(C)
    X = synth.uniform_matrix(A.n_cols, k, seed=k)
    Xd = torch.from_numpy(X.astype(NP[dtype])).cuda()
    Y1 = M.spmm(Xd).cpu().numpy()
    Y2 = M.spmm(Xd).cpu().numpy()
    assert np.array_equal(Y1, Y2)                                      # deterministic, counters reset
    Y_ref, aY = oracle.csr_spmm(A.rowptr, A.col, rounded_values(A.val, dtype), X.astype(NP[dtype]).astype(np.float64))
    assert_within_bound(Y1.ravel(), Y_ref.ravel(), aY.ravel(), TAU[dtype], f"tiles k={k} G={G} {order}")


def test_spmm_tiles_strided_quantized_and_workspace():
    import ctypes
    from paper_1012_2270_gb300 import _lib as L
    from paper_1012_2270_gb300.rgcsr import _ptr, _stream_ptr
    A = synth.power_law(20_000, seed=6)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=32, dtype=torch.float64,
                             row_order="descending")
    Q = M.quantized("bf16").tile_groups(32)
    q, s = oracle.quantize_rows(A.rowptr, A.val, oracle.BF16)
    deq = oracle.dequantized_values(A.rowptr, q, s, oracle.BF16)
    wide = synth.uniform_matrix(A.n_cols, 9, seed=2).astype(np.float32)
    Xd = torch.from_numpy(wide).cuda()[:, 1:7]                          # k = 6, unaligned rows
    Yw = torch.full((A.n_rows, 8), 3.0, device="cuda")
    Q.spmm(Xd, out=Yw[:, 1:7])
    assert (Yw[:, 0] == 3.0).all() and (Yw[:, 7] == 3.0).all()
    Y_ref, aY = oracle.csr_spmm(A.rowptr, A.col, deq, wide[:, 1:7].astype(np.float64))
    assert_within_bound(Yw[:, 1:7].cpu().numpy().ravel(), Y_ref.ravel(), aY.ravel(), 2e-6, "tiles bf16")
    T = Q._tiles[0]
    assert T.n_partials > 0
    part = torch.empty(T.n_partials * 32 * 6 - 1, device="cuda")
    X = torch.zeros(A.n_cols, 6, device="cuda")
    Y = torch.empty(A.n_rows, 6, device="cuda")
    st = L.lib().rgcsr_spmm_tiles(ctypes.byref(Q.s), ctypes.byref(T), 6, _ptr(X), 6, _ptr(Y), 6, _ptr(part),
                                  part.numel(), _stream_ptr())
    assert st == L.RGCSR_ERR_WORKSPACE


@pytest.mark.parametrize("k", [4, 8, 32])
def test_spmm_tiles_full_size_b(k):
    A = synth.workload_b()
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(np.float32), A.n_cols, group_size=32,
                             dtype=torch.float32, row_order="descending").tile_groups(64)
    X = synth.uniform_matrix(A.n_cols, k, seed=k)
    check(A, M, "f32", X, TAU["f32"])
