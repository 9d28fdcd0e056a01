"""GPU parity of reduced-precision value storage (bf16 / fp16 values with a
per-row power-of-two float scale) against the oracle: scales and quantised
bits bit-exact slot by slot, padding +0; SpMV within 2e-6*|A||x| of the
oracle on the dequantised values (kernel error) and within 1e-2*|A||x| of
the original FP64 product (total error)."""
import numpy as np
import pytest
import torch

import oracle
from helpers import assert_within_bound
from paper_1012_2270_gb300 import synth
from paper_1012_2270_gb300 import _lib as L
from paper_1012_2270_gb300.rgcsr import RgCSRMatrix

pytestmark = pytest.mark.gpu

NP = {"f32": np.float32, "f64": np.float64}
TT = {"f32": torch.float32, "f64": torch.float64}
FMT = {"bf16": oracle.BF16, "f16": oracle.F16}


def bits16(t):
    return t.cpu().view(torch.int16).numpy().view(np.uint16)


def check(A, src, fmt, x, G=32, kernels=({}, {"kernel": L.KERNEL_SPLIT}, {"kernel": L.KERNEL_LEAN})):
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[src]), A.n_cols, group_size=G,
                             dtype=TT[src], keep_slot_map=True)
    Q = M.quantized(fmt)
    stored = A.val.astype(NP[src]).astype(np.float64)
    q_ref, s_ref = oracle.quantize_rows(A.rowptr, stored, FMT[fmt])
    assert np.array_equal(Q.row_scale.cpu().numpy(), s_ref)
    s2c = M.slot_to_csr.cpu().numpy()
    qv = bits16(Q.values)
    real = s2c >= 0
    assert np.array_equal(qv[real], q_ref[s2c[real]])
    assert (qv[~real] == 0).all()
    deq = oracle.dequantized_values(A.rowptr, q_ref, s_ref, FMT[fmt])
    x32 = x.astype(np.float32)
    y_deq, a_deq = oracle.csr_spmv(A.rowptr, A.col, deq, x32.astype(np.float64))
    y_orig, a_orig = oracle.csr_spmv(A.rowptr, A.col, A.val, x)
    xd = torch.from_numpy(x32).cuda()
    if G == 32:
        kernels = tuple(kernels) + tuple({"kernel": L.KERNEL_LEAN, "variant": v} for v in (1, 2, 4, 5, 6, 7, 8, 9))   # vector loads
        if A.n_rows >= 32:                                  # bulk-copy ring, several groups per copy
            kernels = kernels + tuple({"kernel": L.KERNEL_TMA, "variant": v} for v in (4, 5, 6))
    for kw in kernels:
        y = Q.spmv(xd, **kw).cpu().numpy()
        assert_within_bound(y, y_deq, a_deq, 2e-6, f"{A.name} {fmt} kernel error {kw}")
        assert_within_bound(y, y_orig, a_orig, 1e-2, f"{A.name} {fmt} total error {kw}")
    return Q


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
@pytest.mark.parametrize("src", ["f64", "f32"])
def test_quantize_ragged_wide_dynamic_range(fmt, src):
    rng = np.random.default_rng(3)
    n = 2011
    Ls = rng.integers(0, 40, n)
    Ls[[7, 900]] = [1500, 700]
    A = synth.random_csr(n, 3000, Ls, seed=3)
    # magnitudes spread over 2^-20 .. 2^20 inside rows, some rows all zero
    A.val = A.val * 2.0 ** rng.integers(-20, 21, A.nnz)
    A.val[A.rowptr[10]:A.rowptr[12]] = 0.0
    check(A, src, fmt, synth.uniform_vector(3000, seed=1))


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_quantize_group_sizes_and_empty(fmt):
    rng = np.random.default_rng(4)
    A = synth.random_csr(500, 200, rng.integers(0, 12, 500), seed=4)
    for G in (1, 8, 33, 64):
        check(A, "f64", fmt, synth.uniform_vector(200, seed=2), G=G)
    E = synth.random_csr(40, 10, np.zeros(40, np.int64))
    Q = check(E, "f32", fmt, np.zeros(10))
    assert (Q.row_scale.cpu() == 1.0).all()


def test_laplacian_values_are_exact_in_bf16():
    # 6 and -1 with scale 8: q = 0.75, -0.125, exact in bfloat16
    A = synth.laplacian_3d(16)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, dtype=torch.float64)
    Q = M.quantized("bf16")
    assert (Q.row_scale.cpu() == 8.0).all()
    x = synth.uniform_vector(A.n_cols, seed=0).astype(np.float32)
    y = Q.spmv(torch.from_numpy(x).cuda()).cpu().numpy()
    y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, A.val, x.astype(np.float64))
    assert_within_bound(y, y_ref, absy, 2e-6, "exact values")


@pytest.mark.parametrize("name", ["a", "b"])
@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_quantized_full_size(name, fmt):
    A = {"a": synth.workload_a, "b": synth.workload_b}[name]()
    check(A, "f64", fmt, synth.uniform_vector(A.n_cols, seed=0), kernels=({},))
