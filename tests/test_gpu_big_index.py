"""A matrix with more than 2^31 stored slots: 2^26 rows of 33 entries each
(2,214,592,512 slots, about 18 GB of slabs in FP32), so that the group
pointers and every slab offset of the last two million rows lie past the
32-bit range.  The conversion is checked against the closed form of the
Sec. 3.4 layout on sampled groups and slots (the closed form itself is
pinned against the oracle's layout on a small case in test_host_logic.py),
and the SpMV kernels against the CPU oracle on sampled rows (the oracle
computes each sampled row from its entries and the full x); likewise BF16
storage and the three SpMM kernels with four right-hand sides."""
import numpy as np
import pytest
import torch

import oracle
from paper_1012_2270_gb300 import synth
from paper_1012_2270_gb300 import _lib as L
from paper_1012_2270_gb300.rgcsr import RgCSRMatrix

pytestmark = pytest.mark.gpu

N = 1 << 26
LEN = 33
G = 32
SLAB = G * LEN                              # slots per group
FIRST_PAST = (2**31 // SLAB + 1) * G        # first row whose slots all lie past 2^31


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1012_2270_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def test_slots_past_2_pow_31():
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < (48 << 30):
        pytest.skip("needs 48 GB of free device memory")
    rowptr, col, val = synth.uniform_rows_device(N, LEN, N)
    M = RgCSRMatrix.from_csr(rowptr, col, val, N, group_size=G, dtype=torch.float32)
    del rowptr, col, val
    torch.cuda.empty_cache()
    nnz = N * LEN
    assert nnz > 2**31 and M.s.nnz == nnz and M.s.n_stored == nnz and M.s.max_row_len == LEN

    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([np.arange(64), np.arange(N - 64, N), rng.integers(0, N, 256),
                                     rng.integers(FIRST_PAST, N, 256), np.arange(FIRST_PAST - 40, FIRST_PAST + 40)]))
    # layout (Sec. 3.4) in closed form: gp[g] = SLAB g, slot j of row i at gp[i // G] + G j + i % G
    groups = np.unique(rows // G)
    gp = M.group_ptr[torch.from_numpy(groups).cuda()].cpu().numpy()
    assert np.array_equal(gp, SLAB * groups)
    assert int(M.group_ptr[-1]) == nnz
    assert bool((M.row_lengths == LEN).all())
    cols_ref, vals_ref = synth.uniform_rows_entries(rows, LEN, N)
    slots = (SLAB * (rows // G))[:, None] + G * np.arange(LEN)[None, :] + (rows % G)[:, None]
    assert slots[rows >= FIRST_PAST].min() > 2**31
    s_t = torch.from_numpy(slots.reshape(-1)).cuda()
    assert np.array_equal(M.columns[s_t].cpu().numpy(), cols_ref.reshape(-1))
    assert np.array_equal(M.values[s_t].cpu().numpy().astype(np.float64), vals_ref.reshape(-1))

    # SpMV: each kernel family on the sampled rows, within 2e-6 |A||x|
    x = synth.uniform_x(N)
    sub_rowptr = np.arange(len(rows) + 1, dtype=np.int64) * LEN
    y_ref, absy = oracle.csr_spmv(sub_rowptr, cols_ref.reshape(-1), vals_ref.reshape(-1), x.astype(np.float64))
    xd = torch.from_numpy(x).cuda()
    r_t = torch.from_numpy(rows).cuda()

    def check(y, what):
        yr = y[r_t].cpu().numpy().astype(np.float64)
        err = np.abs(yr - y_ref)
        assert (err <= 2e-6 * absy).all(), (what, float(err.max()))

    for kw in ({}, dict(kernel=L.KERNEL_LEAN), dict(kernel=L.KERNEL_SPLIT),
               dict(kernel=L.KERNEL_LEAN, variant=1), dict(kernel=L.KERNEL_TMA, variant=2)):
        check(M.spmv(xd, **kw), kw)
    # BF16 storage: the values k/16, |k| <= 8, are exact in bfloat16 after the
    # power-of-two row scale, so the dequantised matrix is the matrix itself
    Q = M.quantized("bf16")
    check(Q.spmv(xd), "bf16")
    del Q

    # SpMM, k = 4: thread per row, lanes per row, then (below) group tiles
    k = 4
    Xh = np.stack([synth.uniform_x(N, shift=3 * c) for c in range(k)], axis=1)
    refs = [oracle.csr_spmv(sub_rowptr, cols_ref.reshape(-1), vals_ref.reshape(-1), Xh[:, c].astype(np.float64))
            for c in range(k)]
    Xd = torch.from_numpy(Xh).cuda()
    del Xh

    def check_mm(Y, what):
        Yr = Y[r_t].cpu().numpy().astype(np.float64)
        for c, (yc, ac) in enumerate(refs):
            err = np.abs(Yr[:, c] - yc)
            assert (err <= 2e-6 * ac).all(), (what, c, float(err.max()))

    check_mm(M.spmm(Xd, rows=False), "spmm thread per row")
    check_mm(M.spmm(Xd, rows=True), "spmm lanes per row")
    M.tile_groups(64)
    check(M.spmv(xd), "tiles")
    check_mm(M.spmm(Xd), "spmm tiles")
    del M, Xd
    torch.cuda.empty_cache()
