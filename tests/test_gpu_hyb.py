"""GPU parity of the HYB (ELL + COO) comparator against the oracle: layout
bit-exact for explicit and automatic ELL widths, SpMV within tau*|A||x|."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TAU, assert_within_bound, rounded_values
from paper_1012_2270_gb300 import synth
from paper_1012_2270_gb300.rgcsr import HybMatrix

pytestmark = pytest.mark.gpu

NP = {"f32": np.float32, "f64": np.float64}
TT = {"f32": torch.float32, "f64": torch.float64}


def check(A, dtype, width):
    H = HybMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols,
                           ell_width=width, dtype=TT[dtype])
    vb = 8 if dtype == "f64" else 4
    K1 = width if width >= 0 else oracle.hyb_choose_ell_width(A.rowptr, vb, 4)
    assert H.ell_width == K1
    lay = oracle.hyb_layout(A.rowptr, A.col, A.val.astype(NP[dtype]), K1)
    assert H.nnz_coo == lay.coo_row.size
    ui = np.uint64 if dtype == "f64" else np.uint32
    assert np.array_equal(H.ell_col.cpu().numpy(), lay.ell_col)
    assert np.array_equal(H.ell_val.cpu().numpy().view(ui), lay.ell_val.view(ui))
    assert np.array_equal(H.coo_row.cpu().numpy(), lay.coo_row)
    assert np.array_equal(H.coo_col.cpu().numpy(), lay.coo_col)
    assert np.array_equal(H.coo_val.cpu().numpy().view(ui), lay.coo_val.view(ui))
    x = synth.uniform_vector(A.n_cols, seed=9)
    y = H.spmv(torch.from_numpy(x.astype(NP[dtype])).cuda()).cpu().numpy()
    y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, rounded_values(A.val, dtype), rounded_values(x, dtype))
    assert_within_bound(y, y_ref, absy, TAU[dtype], f"hyb {A.name} {dtype} K1={K1}")
    return H


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("width", [-1, 0, 1, 3, 17, 64])
def test_hyb_ragged(dtype, width):
    rng = np.random.default_rng(abs(width) + 1)
    L = rng.integers(0, 30, 3000)
    L[[10, 2000, 2001, 2002]] = [2500, 900, 901, 5]
    A = synth.random_csr(3000, 4000, L, seed=3)
    check(A, dtype, width)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_hyb_laplacian_and_empty(dtype):
    check(synth.workload_small_laplacian(), dtype, -1)
    check(synth.random_csr(50, 10, np.zeros(50, np.int64)), dtype, -1)


@pytest.mark.parametrize("name", ["a", "b", "c"])
def test_hyb_full_size(name):
    A = {"a": synth.workload_a, "b": synth.workload_b, "c": synth.workload_c}[name]()
    for dtype in ("f32", "f64"):
        vb = 8 if dtype == "f64" else 4
        H = HybMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, dtype=TT[dtype])
        if name != "b":                 # the oracle's direct rule is O(n * max_len)
            assert H.ell_width == oracle.hyb_choose_ell_width(A.rowptr, vb, 4)
        assert H.nnz_coo == oracle.hyb_coo_count(A.rowptr, H.ell_width)
        x = synth.uniform_vector(A.n_cols, seed=0)
        y = H.spmv(torch.from_numpy(x.astype(NP[dtype])).cuda()).cpu().numpy()
        y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, rounded_values(A.val, dtype), rounded_values(x, dtype))
        assert_within_bound(y, y_ref, absy, TAU[dtype], f"hyb {name} {dtype}")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("width", [-1, 0, 3])
@pytest.mark.parametrize("k", [1, 3, 4, 8, 13, 32, 40])
def test_hyb_spmm(dtype, width, k):
    rng = np.random.default_rng(k + width)
    Ls = rng.integers(0, 30, 1200)
    Ls[[4, 600]] = [2000, 700]
    A = synth.random_csr(1200, 2500, Ls, seed=k)
    H = HybMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, ell_width=width, dtype=TT[dtype])
    X = synth.uniform_matrix(A.n_cols, k, seed=k).astype(NP[dtype])
    Y = H.spmm(torch.from_numpy(X).cuda()).cpu().numpy()
    Y_ref, aY = oracle.csr_spmm(A.rowptr, A.col, rounded_values(A.val, dtype), X.astype(np.float64))
    assert_within_bound(Y.ravel(), Y_ref.ravel(), aY.ravel(), TAU[dtype], f"hyb spmm k={k} K1={H.ell_width}")


def test_hyb_spmm_strided_and_full_size_b():
    A = synth.workload_b()
    H = HybMatrix.from_csr(A.rowptr, A.col, A.val.astype(np.float32), A.n_cols, dtype=torch.float32)
    wide = synth.uniform_matrix(A.n_cols, 10, seed=1).astype(np.float32)
    Xd = torch.from_numpy(wide).cuda()[:, 1:9]                        # k = 8, row stride 10
    Yw = torch.full((A.n_rows, 10), 2.0, device="cuda")
    H.spmm(Xd, out=Yw[:, 1:9])
    assert (Yw[:, 0] == 2.0).all() and (Yw[:, 9] == 2.0).all()
    Y_ref, aY = oracle.csr_spmm(A.rowptr, A.col, rounded_values(A.val, "f32"), wide[:, 1:9].astype(np.float64))
    assert_within_bound(Yw[:, 1:9].cpu().numpy().ravel(), Y_ref.ravel(), aY.ravel(), TAU["f32"], "hyb spmm b")
