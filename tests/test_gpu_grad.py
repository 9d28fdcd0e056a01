"""GPU parity of the backward pass: the stable CSR transposition bit-exact
against the oracle's counting sort; gradients of loss = ||A X||^2 with
respect to values and X against the oracle's closed form (elementwise,
scaled by the absolute-value product); FP64 central finite differences on
the n = 4,096 Laplacian; matrix (b) with a batch of 8 right-hand sides."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from helpers import TAU, assert_within_bound, rounded_values
from paper_1012_2270_gb300 import synth
from paper_1012_2270_gb300 import _lib as L
from paper_1012_2270_gb300.autograd import SparseOperator, spmm
from paper_1012_2270_gb300.rgcsr import RgCSRMatrix, _ptr, csr_struct, _stream_ptr

pytestmark = pytest.mark.gpu

NP = {"f32": np.float32, "f64": np.float64}
TT = {"f32": torch.float32, "f64": torch.float64}


def gpu_transpose(A):
    rp = torch.from_numpy(A.rowptr).cuda()
    col = torch.from_numpy(A.col).cuda()
    val = torch.from_numpy(A.val).cuda()
    nb = L.lib().rgcsr_transpose_workspace_bytes(A.nnz, A.n_rows, A.n_cols)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    trp = torch.empty(A.n_cols + 1, dtype=torch.int64, device="cuda")
    tc = torch.empty(A.nnz, dtype=torch.int32, device="cuda")
    perm = torch.empty(A.nnz, dtype=torch.int64, device="cuda")
    tv = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
    L.call("rgcsr_csr_transpose", ctypes.byref(csr_struct(rp, col, val, A.n_cols)), _ptr(trp), _ptr(tc),
           _ptr(perm), _ptr(tv), _ptr(ws), nb, _stream_ptr())
    return trp.cpu().numpy(), tc.cpu().numpy(), perm.cpu().numpy(), tv.cpu().numpy()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_transpose_bit_exact(seed):
    rng = np.random.default_rng(seed)
    n, m = [(3000, 2000), (1, 700), (5000, 300)][seed]
    Ls = rng.integers(0, min(m, 60) + 1, n)
    A = synth.random_csr(n, m, Ls, seed=seed)
    trp, tc, perm = oracle.csr_transpose(A.rowptr, A.col, m)
    g = gpu_transpose(A)
    assert np.array_equal(g[0], trp) and np.array_equal(g[1], tc) and np.array_equal(g[2], perm)
    assert np.array_equal(g[3], A.val[perm])


def test_transpose_many_columns_and_empty():
    # more than 2^16 columns (three radix passes), empty rows and columns
    rng = np.random.default_rng(5)
    A = synth.random_csr(20000, 300000, rng.integers(0, 8, 20000), seed=5)
    trp, tc, perm = oracle.csr_transpose(A.rowptr, A.col, A.n_cols)
    g = gpu_transpose(A)
    assert np.array_equal(g[0], trp) and np.array_equal(g[1], tc) and np.array_equal(g[2], perm)
    E = synth.random_csr(10, 7, np.zeros(10, np.int64))
    assert gpu_transpose(E)[0].tolist() == [0] * 8


def abs_bounds(A, vals, X, G):
    """|A^T||G| and sum_b |G[row,b]||X[col,b]| from the oracle."""
    trp, tc, perm = oracle.csr_transpose(A.rowptr, A.col, A.n_cols)
    dX_abs, _ = oracle.csr_spmm(trp, tc, np.abs(vals)[perm], np.abs(G))
    _, dval_abs = oracle.spmm_grads(A.rowptr, A.col, vals, np.abs(X), np.abs(G), A.n_cols)
    return dX_abs, dval_abs


def check_grads(A, dtype, k, group_size=32, seed=0, **schedule):
    vals = rounded_values(A.val, dtype)
    X = synth.uniform_matrix(A.n_cols, k, seed=seed).astype(NP[dtype]).astype(np.float64)
    op = SparseOperator(A.rowptr, A.col, A.n_cols, dtype=TT[dtype], group_size=group_size, **schedule)
    v = torch.tensor(vals, dtype=TT[dtype], device="cuda", requires_grad=True)
    Xt = torch.tensor(X, dtype=TT[dtype], device="cuda", requires_grad=True)
    Y = spmm(op, v, Xt)
    loss = (Y * Y).sum()
    loss.backward()
    # the oracle's gradient for the upstream gradient the GPU actually used
    Gy = (2.0 * Y.detach()).double().cpu().numpy()
    dX_ref, dval_ref = oracle.spmm_grads(A.rowptr, A.col, vals, X, Gy, A.n_cols)
    dX_abs, dval_abs = abs_bounds(A, vals, X, Gy)
    assert_within_bound(Xt.grad.double().cpu().numpy().ravel(), dX_ref.ravel(), dX_abs.ravel(),
                        TAU[dtype], f"dX {A.name} {dtype}")
    assert_within_bound(v.grad.double().cpu().numpy(), dval_ref, dval_abs, TAU[dtype],
                        f"dval {A.name} {dtype}")
    return op


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("k", [1, 3, 8])
def test_grads_ragged(dtype, k):
    rng = np.random.default_rng(k)
    Ls = rng.integers(0, 25, 1200)
    Ls[[2, 600]] = [900, 300]
    A = synth.random_csr(1200, 1500, Ls, seed=k)
    check_grads(A, dtype, k)
    check_grads(A, dtype, k, group_size=8)
    check_grads(A, dtype, k, group_size=32, row_order="descending", tiles=16)
    check_grads(A, dtype, k, group_size=1, long_rows=(16, 64))


def test_values_refresh_between_calls():
    A = synth.workload_small_laplacian()
    op = SparseOperator(A.rowptr, A.col, A.n_cols, dtype=torch.float64)
    x = torch.from_numpy(synth.uniform_vector(A.n_cols, 0)).cuda()
    for scale in (1.0, -2.5, 0.0):
        v = torch.from_numpy(A.val * scale).cuda()
        y = spmm(op, v, x).cpu().numpy()
        y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, A.val * scale, x.cpu().numpy())
        assert_within_bound(y, y_ref, absy, 1e-12, f"scale {scale}")


def test_fp64_finite_differences_laplacian():
    A = synth.workload_small_laplacian()
    op = SparseOperator(A.rowptr, A.col, A.n_cols, dtype=torch.float64)
    rng = np.random.default_rng(0)
    vals = A.val + 0.1 * rng.standard_normal(A.nnz)
    X = synth.uniform_matrix(A.n_cols, 2, seed=3)
    v = torch.tensor(vals, device="cuda", requires_grad=True)
    Xt = torch.tensor(X, device="cuda", requires_grad=True)
    loss = (spmm(op, v, Xt) ** 2).sum()
    loss.backward()

    def f(vv, XX):
        with torch.no_grad():
            return float((spmm(op, vv, XX) ** 2).sum())
    vt, Xd = torch.tensor(vals, device="cuda"), torch.tensor(X, device="cuda")
    # the loss is quadratic in every value and every entry of X, so central
    # differences carry no truncation error; a moderate step keeps the
    # cancellation error of the O(1e4) loss well below the tolerance
    for p in rng.integers(0, A.nnz, 40):
        h = 1e-3 * max(1.0, abs(vals[p]))
        vp, vm = vt.clone(), vt.clone()
        vp[p] += h
        vm[p] -= h
        fd = (f(vp, Xd) - f(vm, Xd)) / (2 * h)
        g = float(v.grad[p])
        assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (p, fd, g)
    for idx in [(0, 0), (A.n_cols - 1, 1), (2048, 0), (63, 1)]:
        h = 1e-3 * max(1.0, abs(X[idx]))
        Xp, Xm = Xd.clone(), Xd.clone()
        Xp[idx] += h
        Xm[idx] -= h
        fd = (f(vt, Xp) - f(vt, Xm)) / (2 * h)
        g = float(Xt.grad[idx])
        assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (idx, fd, g)
    # and the oracle's closed form agrees with the GPU in FP64
    Gy = 2.0 * oracle.csr_spmm(A.rowptr, A.col, vals, X)[0]
    dX_ref, dval_ref = oracle.spmm_grads(A.rowptr, A.col, vals, X, Gy, A.n_cols)
    assert np.allclose(v.grad.cpu().numpy(), dval_ref, rtol=1e-10, atol=1e-10)
    assert np.allclose(Xt.grad.cpu().numpy(), dX_ref, rtol=1e-10, atol=1e-10)


def test_gradcheck_tiny():
    A = synth.random_csr(40, 30, np.random.default_rng(1).integers(0, 8, 40), seed=1)
    op = SparseOperator(A.rowptr, A.col, A.n_cols, dtype=torch.float64, group_size=4)
    v = torch.tensor(A.val, device="cuda", requires_grad=True)
    X = torch.tensor(synth.uniform_matrix(30, 3, seed=2), device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda vv, XX: spmm(op, vv, XX), (v, X), eps=1e-6, atol=1e-8)


def test_grads_full_size_b_batch8():
    A = synth.workload_b()
    check_grads(A, "f32", 8)
    check_grads(A, "f32", 8, row_order="descending", tiles=64)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("G,order,k", [(32, None, 1), (32, "descending", 5), (7, None, 8), (1, None, 3)])
def test_bwd_values_from_rgcsr(dtype, G, order, k):
    # rgcsr_spmv_bwd_values: the value gradient straight from the RgCSR slabs
    rng = np.random.default_rng(k + G)
    Ls = rng.integers(0, 25, 900)
    Ls[[3, 500]] = [700, 260]
    A = synth.random_csr(900, 1100, Ls, seed=k)
    vals = rounded_values(A.val, dtype)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=G, dtype=TT[dtype],
                             keep_slot_map=True, row_order=order)
    X = synth.uniform_matrix(A.n_cols, k, seed=1).astype(NP[dtype]).astype(np.float64)
    Gy = synth.uniform_matrix(A.n_rows, k, seed=2).astype(NP[dtype]).astype(np.float64)
    dval = M.value_grad(torch.tensor(Gy, dtype=TT[dtype], device="cuda"),
                        torch.tensor(X, dtype=TT[dtype], device="cuda")).double().cpu().numpy()
    _, dval_ref = oracle.spmm_grads(A.rowptr, A.col, vals, X, Gy, A.n_cols)
    _, dval_abs = abs_bounds(A, vals, X, Gy)
    assert_within_bound(dval, dval_ref, dval_abs, TAU[dtype], f"bwd values G={G} {order}")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("schedule", [{}, {"row_order": "descending", "tiles": 16}])
def test_values_reloaded_only_when_they_change(dtype, schedule):
    # the operator gathers values into A (forward) or A^T (backward) only
    # when the values tensor changed: products stay right when values are
    # updated in place, when another tensor is used, and when a backward
    # runs after a forward with other values; with and without a row order
    # and group tiles on A and A^T
    rng = np.random.default_rng(9)
    A = synth.random_csr(700, 500, rng.integers(0, 30, 700), seed=9)
    op = SparseOperator(A.rowptr, A.col, A.n_cols, dtype=TT[dtype], **schedule)
    X = synth.uniform_matrix(A.n_cols, 3, seed=4).astype(NP[dtype])
    Xt = torch.tensor(X, device="cuda")

    def expect(vals):
        y, absy = oracle.csr_spmm(A.rowptr, A.col, vals.astype(np.float64), X.astype(np.float64))
        return y, absy

    v1 = torch.tensor(A.val.astype(NP[dtype]), device="cuda")
    with torch.no_grad():
        y = spmm(op, v1, Xt)
        assert_within_bound(y.cpu().numpy(), *expect(A.val.astype(NP[dtype])), TAU[dtype], "first")
        y = spmm(op, v1, Xt)                                   # unchanged: no reload, same product
        assert_within_bound(y.cpu().numpy(), *expect(A.val.astype(NP[dtype])), TAU[dtype], "again")
        v1.mul_(-2.0)                                          # in place
        y = spmm(op, v1, Xt)
        assert_within_bound(y.cpu().numpy(), *expect(-2.0 * A.val.astype(NP[dtype])), TAU[dtype], "in place")
        v1.data[17] = 5.0                                      # through .data: no version change, still seen
        vals = -2.0 * A.val.astype(NP[dtype])
        vals[17] = 5.0
        y = spmm(op, v1, Xt)
        assert_within_bound(y.cpu().numpy(), *expect(vals), TAU[dtype], ".data")
        # unchanged values are not gathered again: overwrite the matrix's own
        # slab, and a product with the same values keeps the overwritten slab
        op.A.values.zero_()
        y = spmm(op, v1, Xt)
        assert not y.any()
        op.load_values(v1, force=True)
        y = spmm(op, v1, Xt)
        assert_within_bound(y.cpu().numpy(), *expect(vals), TAU[dtype], "forced reload")
    # backward of a product with v2 after a forward with v3: dX uses v2
    v2 = torch.tensor((0.5 * A.val).astype(NP[dtype]), device="cuda", requires_grad=True)
    v3 = torch.tensor((3.0 * A.val).astype(NP[dtype]), device="cuda")
    Xg = torch.tensor(X, device="cuda", requires_grad=True)
    Y = spmm(op, v2, Xg)
    with torch.no_grad():
        spmm(op, v3, Xt)
    Gy = torch.ones_like(Y)
    Y.backward(Gy)
    vals2 = (0.5 * A.val).astype(NP[dtype]).astype(np.float64)
    trp, tc, perm = oracle.csr_transpose(A.rowptr, A.col, A.n_cols)
    dX_ref, dX_abs = oracle.csr_spmm(trp, tc, vals2[perm], np.ones((A.n_rows, 3)))
    assert_within_bound(Xg.grad.cpu().numpy(), dX_ref, dX_abs, TAU[dtype], "dX after other values")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("offset", [0, 1])
def test_value_hash_sees_every_change(dtype, offset):
    # the refresh decision itself (rgcsr_gather_values_if_changed's state
    # record, word 1 bit 1 = changed by this call): a change of one element
    # anywhere -- first, last (in the zero-filled last word when n is odd),
    # an interior one, a sign, a single low bit -- and a swap of two unequal
    # elements are all seen; an unchanged tensor is not.  offset = 1 starts
    # the values off a 16-byte boundary (the word-by-word path).
    rng = np.random.default_rng(21)
    lengths = rng.integers(1, 9, 301)
    lengths[0] += 1 - lengths.sum() % 2      # an odd count of values
    A = synth.random_csr(301, 250, lengths, seed=21)
    assert A.nnz % 2 == 1
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, dtype=TT[dtype],
                             keep_slot_map=True)
    buf = torch.tensor(np.r_[np.zeros(offset), A.val].astype(NP[dtype]), device="cuda")
    v = buf[offset:]
    n = v.numel()
    state = torch.zeros(L.VALUES_STATE_BYTES // 8, dtype=torch.int64, device="cuda")

    def changed():
        L.call("rgcsr_gather_values_if_changed", ctypes.byref(M.s), _ptr(v), n, _ptr(M.slot_to_csr),
               _ptr(state), _stream_ptr())
        return bool(state[1].item() & 2)

    assert changed()                         # first call: the record held nothing
    assert not changed()
    ints = v.view(torch.int32 if dtype == "f32" else torch.int64)
    for i in (0, 1, n // 2, n - 2, n - 1):
        old = v[i].item()
        v[i] = -old
        assert changed(), i
        assert not changed(), i
        ints[i] ^= 1                         # the lowest bit
        assert changed(), i
        v[i] = old
        assert changed(), i
    for i, j in ((3, n - 4), (4, 5), (4, 4 + 8 // v.element_size())):
        # far apart; neighbours; the two 8-byte words of one 16-byte pack
        assert v[i].item() != v[j].item()
        vi, vj = v[i].item(), v[j].item()
        v[i], v[j] = vj, vi
        assert changed(), (i, j)
        assert not changed()
    v.mul_(2.0)                              # every element at once
    assert changed()
    v.neg_()                                 # every sign bit at once
    assert changed()
    assert not changed()
    ints.add_(1)                             # every lowest bit at once
    assert changed()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("k,ld", [(2, 2), (4, 4), (8, 8), (8, 12), (4, 5), (3, 3)])
def test_sampled_dot_against_oracle(dtype, k, ld):
    # rgcsr_sampled_dot with 16-byte row loads (k = 2 for FP64, 4, 8 with
    # aligned rows) and the scalar path (odd strides, k = 3): the same sums,
    # in increasing b, as the oracle's value gradient
    rng = np.random.default_rng(k * 10 + ld)
    A = synth.random_csr(500, 400, rng.integers(0, 30, 500), seed=k)
    rows = torch.tensor(np.repeat(np.arange(A.n_rows), np.diff(A.rowptr)).astype(np.int32), device="cuda")
    cols = torch.tensor(A.col, device="cuda")
    Gm = synth.uniform_matrix(A.n_rows, ld, seed=1).astype(NP[dtype])
    Xm = synth.uniform_matrix(A.n_cols, ld, seed=2).astype(NP[dtype])
    Gt, Xt = torch.tensor(Gm, device="cuda"), torch.tensor(Xm, device="cuda")
    out = torch.empty(A.nnz, dtype=TT[dtype], device="cuda")
    L.call("rgcsr_sampled_dot", A.nnz, k, _ptr(rows), _ptr(cols), _ptr(Gt), ld, _ptr(Xt), ld, _ptr(out),
           L.F64 if dtype == "f64" else L.F32, _stream_ptr())
    _, ref = oracle.spmm_grads(A.rowptr, A.col, A.val, Xm[:, :k].astype(np.float64),
                               Gm[:, :k].astype(np.float64), A.n_cols)
    _, absref = oracle.spmm_grads(A.rowptr, A.col, A.val, np.abs(Xm[:, :k]).astype(np.float64),
                                  np.abs(Gm[:, :k]).astype(np.float64), A.n_cols)
    assert_within_bound(out.cpu().numpy(), ref, absref, TAU[dtype], f"sampled dot k={k} ld={ld}")
