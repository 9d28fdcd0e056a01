"""GPU parity of row-ordered RgCSR (Sec. 4.4.2, Table 7: the groups are
formed over the rows sorted by length, longest first, or over any given
permutation) against the CPU oracle: the device descending order equals the
oracle's (bit-exact), the layout of P A is bit-exact, every kernel returns
y in the CSR's own row order within tau*|A||x|, and an invalid permutation
is rejected."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from helpers import TAU, assert_within_bound, rounded_values
from paper_1012_2270_gb300 import synth
from paper_1012_2270_gb300 import _lib as L
from paper_1012_2270_gb300.rgcsr import RgCSRMatrix, csr_struct, _ptr, _stream_ptr

pytestmark = pytest.mark.gpu

NP = {"f32": np.float32, "f64": np.float64}
TT = {"f32": torch.float32, "f64": torch.float64}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1012_2270_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def kernels(M):
    out = [dict(), dict(kernel=L.KERNEL_SPLIT), dict(kernel=L.KERNEL_LEAN)]
    if M.group_size <= 1024:
        out.append(dict(kernel=L.KERNEL_PAPER))
    if M.group_size == 32 and M.shape[0] >= 32:
        out += [dict(kernel=L.KERNEL_TMA, variant=v) for v in range(4)]
    return out


def check_layout(M, A, dtype, G, perm):
    lay = oracle.rgcsr_layout(A.rowptr, A.col, A.val.astype(NP[dtype]), G, row_order=perm)
    assert np.array_equal(M.row_perm.cpu().numpy(), perm)
    assert M.n_stored == lay.n_stored
    assert np.array_equal(M.row_lengths.cpu().numpy(), lay.row_lengths)
    assert np.array_equal(M.group_ptr.cpu().numpy(), lay.group_ptr)
    assert np.array_equal(M.columns.cpu().numpy(), lay.columns)
    ui = np.uint64 if dtype == "f64" else np.uint32
    assert np.array_equal(M.values.cpu().numpy().view(ui), lay.values.view(ui))
    assert np.array_equal(M.slot_to_csr.cpu().numpy(), lay.slot_to_csr)


def check_spmv(M, A, dtype, x, **kw):
    xd = torch.from_numpy(x.astype(NP[dtype])).cuda()
    y = M.spmv(xd, **kw).cpu().numpy()
    y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, rounded_values(A.val, dtype), rounded_values(x, dtype))
    assert_within_bound(y, y_ref, absy, TAU[dtype], f"{A.name} {dtype} {kw}")


def ragged(n, m, seed):
    rng = np.random.default_rng(seed)
    lengths = rng.integers(0, 30, n)
    lengths[[3, n // 2]] = [500, 90]
    return synth.random_csr(n, m, lengths, seed=seed)


@pytest.mark.parametrize("n", [1, 31, 1000, 70_001])
def test_descending_order_matches_oracle(n):
    A = ragged(n, 600, seed=n) if n > 1 else synth.random_csr(1, 4, np.array([3]), seed=0)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=32, row_order="descending")
    assert np.array_equal(M.row_perm.cpu().numpy(), oracle.descending_order(A.rowptr))


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("G", [1, 3, 32, 64])
@pytest.mark.parametrize("order", ["descending", "random"])
def test_reordered_layout_and_spmv(dtype, G, order):
    A = ragged(1000, 700, seed=G)
    perm = (oracle.descending_order(A.rowptr) if order == "descending"
            else np.random.default_rng(G).permutation(A.n_rows))
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=G,
                             dtype=TT[dtype], keep_slot_map=True,
                             row_order="descending" if order == "descending" else perm)
    check_layout(M, A, dtype, G, perm)
    x = synth.uniform_vector(A.n_cols, seed=2)
    for kw in kernels(M):
        check_spmv(M, A, dtype, x, **kw)
    M.split_long_rows(threshold=16, segment=64)
    check_spmv(M, A, dtype, x)


def test_descending_cuts_padding():
    # Table 7: descending order removes most artificial zeros
    A = synth.power_law(50_000, seed=7)
    plain = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=32)
    desc = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=32, row_order="descending")
    lay = oracle.rgcsr_layout(A.rowptr, A.col, A.val, 32, row_order=oracle.descending_order(A.rowptr))
    assert desc.n_stored == lay.n_stored
    assert desc.n_stored < plain.n_stored
    assert desc.artificial_zero_percent() < 0.05 * plain.artificial_zero_percent()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_reordered_spmm_and_host_path(dtype):
    A = ragged(3000, 2000, seed=11)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=32,
                             dtype=TT[dtype], row_order="descending")
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (A.n_cols, 5)).astype(NP[dtype])
    Y = M.spmm(torch.from_numpy(X).cuda()).cpu().numpy()
    val = rounded_values(A.val, dtype)
    for b in range(5):
        y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, val, X[:, b].astype(np.float64))
        assert_within_bound(Y[:, b], y_ref, absy, TAU[dtype], f"spmm col {b}")
    x = synth.uniform_vector(A.n_cols, seed=4).astype(NP[dtype])
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty(A.n_rows, dtype=TT[dtype]).pin_memory()
    M.spmv_host(xh, yh, torch.empty_like(xh, device="cuda"), torch.empty_like(yh, device="cuda"))
    torch.cuda.synchronize()
    y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, val, x.astype(np.float64))
    assert_within_bound(yh.numpy(), y_ref, absy, TAU[dtype], "host path")


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_reordered_quantized(fmt):
    A = synth.power_law(20_000, seed=5)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=32, dtype=torch.float64,
                             row_order="descending")
    Q = M.quantized(fmt)
    code = oracle.BF16 if fmt == "bf16" else oracle.F16
    q, sc = oracle.quantize_rows(A.rowptr, A.val, code)
    perm = oracle.descending_order(A.rowptr)
    assert np.array_equal(Q.row_scale.cpu().numpy(), sc[perm].astype(np.float32))
    x = synth.uniform_vector(A.n_cols, seed=1).astype(np.float32)
    deq = oracle.dequantized_values(A.rowptr, q, sc, code)
    y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, deq, x.astype(np.float64))
    for kw in (dict(), dict(kernel=L.KERNEL_SPLIT), dict(kernel=L.KERNEL_LEAN)):
        y = Q.spmv(torch.from_numpy(x).cuda(), **kw).cpu().numpy()
        assert_within_bound(y, y_ref, absy, 2e-6, f"{fmt} {kw}")


def test_bad_permutation_rejected():
    A = ragged(100, 600, seed=1)
    for bad in (np.zeros(100, np.int32), np.r_[np.arange(99), 100].astype(np.int32),
                np.r_[np.arange(99), -1].astype(np.int32)):
        with pytest.raises(L.RgCSRError) as e:
            RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=8, row_order=bad)
        assert e.value.status == L.RGCSR_ERR_BAD_PERM
    with pytest.raises(ValueError):
        RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=8, row_order=np.arange(5))


def test_descending_order_workspace_errors():
    A = ragged(100, 600, seed=2)
    rp = torch.from_numpy(A.rowptr).cuda()
    col = torch.from_numpy(A.col).cuda()
    val = torch.from_numpy(A.val).cuda()
    C = csr_struct(rp, col, val, A.n_cols)
    perm = torch.empty(100, dtype=torch.int32, device="cuda")
    need = L.lib().rgcsr_row_order_workspace_bytes(100)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    st = L.lib().rgcsr_descending_order(ctypes.byref(C), _ptr(perm), _ptr(ws), need - 1, _stream_ptr())
    assert st == L.RGCSR_ERR_WORKSPACE
    st = L.lib().rgcsr_descending_order(ctypes.byref(C), None, _ptr(ws), need, _stream_ptr())
    assert st == L.RGCSR_ERR_INVALID_ARG


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_full_size_b_descending(dtype):
    A = synth.workload_b()
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=32,
                             dtype=TT[dtype], row_order="descending")
    perm = oracle.descending_order(A.rowptr)
    assert np.array_equal(M.row_perm.cpu().numpy(), perm)
    lengths = np.diff(A.rowptr)[perm]
    rl, gp = oracle.rgcsr_sizes(np.concatenate([[0], np.cumsum(lengths)]), 32)
    assert np.array_equal(M.row_lengths.cpu().numpy(), rl)
    assert np.array_equal(M.group_ptr.cpu().numpy(), gp)
    x = synth.uniform_vector(A.n_cols, seed=0)
    for kw in kernels(M):
        check_spmv(M, A, dtype, x, **kw)
    M.split_long_rows(threshold=64, segment=256)
    check_spmv(M, A, dtype, x)
