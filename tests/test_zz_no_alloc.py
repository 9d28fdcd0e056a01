"""rgcsr_plan_noalloc -- the plan step for callers that cannot allocate
device memory (they only hold device pointers handed to them, or must not
trigger a device-wide synchronising cudaMalloc/cudaFree) -- gives the same
row lengths, group pointers and sizes as rgcsr_plan with a caller-provided
workspace, on consecutive calls that share its one fixed scratch array, and
refuses matrices whose scratch would exceed that array.

This file is collected last on purpose, and passes alone or after the
other tests (every call looks up the array's device address)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1012_2270_gb300 import build as B
from paper_1012_2270_gb300 import synth
from paper_1012_2270_gb300 import _lib as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    B.build()
    assert torch.cuda.is_available()
    return L.lib()


def csr_on_device(A):
    rp = torch.from_numpy(A.rowptr).cuda()
    col = torch.from_numpy(A.col).cuda()
    val = torch.from_numpy(A.val.astype(np.float32)).cuda()
    c = L.CSR(n_rows=A.n_rows, n_cols=A.n_cols, nnz=A.nnz, row_ptr=rp.data_ptr(),
              row_ptr_type=L.I64T, value_type=L.F32, col_idx=col.data_ptr(),
              values=val.data_ptr())
    return c, (rp, col, val)


def plan_outputs(lib, A, G, noalloc):
    c, keep = csr_on_device(A)
    n_groups = (A.n_rows + G - 1) // G
    rl = torch.full((max(A.n_rows, 1),), -7, dtype=torch.int32, device="cuda")
    gp = torch.full((n_groups + 1,), -7, dtype=torch.int64, device="cuda")
    M = L.Matrix(group_size=G, value_type=L.F32, row_lengths=rl.data_ptr(), group_ptr=gp.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if noalloc:
        st = lib.rgcsr_plan_noalloc(ctypes.byref(c), ctypes.byref(M), stream)
    else:
        nb = lib.rgcsr_plan_workspace_bytes(A.n_rows, G)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        st = lib.rgcsr_plan(ctypes.byref(c), ctypes.byref(M), ctypes.c_void_p(ws.data_ptr()), nb, stream)
    assert st == L.RGCSR_OK, lib.rgcsr_status_string(st)
    torch.cuda.synchronize()
    return (M.n_groups, M.n_stored, M.max_row_len, M.nnz,
            rl.cpu().numpy()[:A.n_rows].copy(), gp.cpu().numpy().copy())


def assert_same(a, b):
    assert a[:4] == b[:4]
    assert np.array_equal(a[4], b[4]) and np.array_equal(a[5], b[5])


def test_noalloc_plan_matches_plan_on_consecutive_calls(lib):
    rng = np.random.default_rng(3)
    L_ = rng.integers(0, 40, 20011)          # partial last group, many scan tiles
    L_[[5, 9000]] = [3000, 1200]
    first = synth.random_csr(20011, 5000, L_, seed=3)
    second = synth.workload_small_laplacian()
    # two calls in a row on different matrices, then the first again: the
    # shared array keeps the previous call's contents and must not leak them
    for A, G in ((first, 32), (second, 32), (first, 7)):
        assert_same(plan_outputs(lib, A, G, noalloc=True), plan_outputs(lib, A, G, noalloc=False))


def test_noalloc_plan_reports_validation_errors(lib):
    A = synth.random_csr(100, 50, np.full(100, 3), seed=1)
    A.col = A.col.copy()
    A.col[10] = 50
    c, keep = csr_on_device(A)
    rl = torch.empty(100, dtype=torch.int32, device="cuda")
    gp = torch.empty(5, dtype=torch.int64, device="cuda")
    M = L.Matrix(group_size=32, value_type=L.F32, row_lengths=rl.data_ptr(), group_ptr=gp.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.rgcsr_plan_noalloc(ctypes.byref(c), ctypes.byref(M), stream) == L.RGCSR_ERR_COL_OOB
    # a valid call afterwards is unaffected by the error left in the array
    B_ = synth.random_csr(100, 50, np.full(100, 3), seed=2)
    assert_same(plan_outputs(lib, B_, 32, noalloc=True), plan_outputs(lib, B_, 32, noalloc=False))


def test_noalloc_plan_rejects_beyond_fixed_maximum(lib):
    # 16,709,632 groups (G = 1) need more scratch than the fixed array holds:
    # refused with RGCSR_ERR_WORKSPACE.  Every buffer is a real device array
    # of the size the call declares (an empty valid CSR), so even a missed
    # check could only touch memory that belongs to the call.
    n = 16_709_632
    assert lib.rgcsr_plan_workspace_bytes(n - 1, 1) <= 65536
    assert lib.rgcsr_plan_workspace_bytes(n, 1) > 65536
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    val = torch.zeros(1, dtype=torch.float32, device="cuda")
    rl = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    gp = torch.full((n + 1,), -7, dtype=torch.int64, device="cuda")
    c = L.CSR(n_rows=n, n_cols=10, nnz=0, row_ptr=rp.data_ptr(), row_ptr_type=L.I64T,
              value_type=L.F32, col_idx=col.data_ptr(), values=val.data_ptr())
    M = L.Matrix(group_size=1, value_type=L.F32, row_lengths=rl.data_ptr(), group_ptr=gp.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.rgcsr_plan_noalloc(ctypes.byref(c), ctypes.byref(M), stream) == L.RGCSR_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert int(rl[0]) == -7 and int(gp[-1]) == -7          # nothing written
