"""GPU parity of the RgCSR path against the CPU oracle, through the C ABI:
conversion bit-exact (row lengths, group pointers, value bits, columns,
slot map), SpMV within tau*|A||x| for every kernel variant, edge cases and
error codes, and the full-size workloads in the benchmark's configuration."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TAU, assert_within_bound, rounded_values
from paper_1012_2270_gb300 import synth
from paper_1012_2270_gb300 import _lib as L
from paper_1012_2270_gb300.rgcsr import HybMatrix, RgCSRMatrix

pytestmark = pytest.mark.gpu

NP = {"f32": np.float32, "f64": np.float64}
TT = {"f32": torch.float32, "f64": torch.float64}
VARIANTS = [dict(), dict(kernel=L.KERNEL_PAPER), dict(kernel=L.KERNEL_SPLIT, x_load=L.XLOAD_PLAIN),
            dict(kernel=L.KERNEL_SPLIT, block_threads=64, split_weight=4), dict(kernel=L.KERNEL_LEAN)]
VARIANTS += [dict(kernel=L.KERNEL_TMA, variant=v) for v in range(0, 7)]
VARIANTS += [dict(kernel=L.KERNEL_LEAN, variant=v) for v in (1, 2, 4, 5, 6, 7, 8)]   # vector loads, G = 32
# the x read paths: texture fetches and plain loads besides the read-only path
VARIANTS += [dict(kernel=k, x_load=xl) for k in (L.KERNEL_PAPER, L.KERNEL_SPLIT, L.KERNEL_LEAN)
             for xl in (L.XLOAD_TEX, L.XLOAD_PLAIN)]


def variants(M):
    """Kernel variants valid for M (the TMA kernel needs G = 32, n >= 32)."""
    out = []
    for kw in VARIANTS:
        if kw.get("kernel") == L.KERNEL_TMA and (M.group_size != 32 or M.shape[0] < 32):
            continue
        if kw.get("kernel") == L.KERNEL_LEAN and kw.get("variant", 0) > 0 and M.group_size != 32:
            continue
        if kw.get("kernel") == L.KERNEL_PAPER and M.group_size > 1024:
            continue
        out.append(kw)
    return out


def device_status():
    import ctypes
    st = ctypes.c_int(-1)
    L.call("rgcsr_get_status", ctypes.byref(st), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st.value


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1012_2270_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def to_gpu_matrix(A, dtype, G, rowptr_i32=False, slot_map=True):
    rp = A.rowptr.astype(np.int32) if rowptr_i32 else A.rowptr
    return RgCSRMatrix.from_csr(rp, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=G,
                                dtype=TT[dtype], keep_slot_map=slot_map)


def check_layout(M, A, dtype, G):
    lay = oracle.rgcsr_layout(A.rowptr, A.col, A.val.astype(NP[dtype]), G)
    assert M.n_stored == lay.n_stored
    assert M.max_row_len == (int(A.row_lengths().max()) if A.n_rows else 0)
    assert np.array_equal(M.row_lengths.cpu().numpy(), lay.row_lengths)
    assert np.array_equal(M.group_ptr.cpu().numpy(), lay.group_ptr)
    assert np.array_equal(M.columns.cpu().numpy(), lay.columns)
    ui = np.uint64 if dtype == "f64" else np.uint32
    assert np.array_equal(M.values.cpu().numpy().view(ui), lay.values.view(ui))
    if M.slot_to_csr is not None:
        assert np.array_equal(M.slot_to_csr.cpu().numpy(), lay.slot_to_csr)


def check_spmv(M, A, dtype, x, **kw):
    xd = torch.from_numpy(x.astype(NP[dtype])).cuda()
    y = M.spmv(xd, **kw).cpu().numpy()
    y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, rounded_values(A.val, dtype),
                                  rounded_values(x, dtype))
    assert_within_bound(y, y_ref, absy, TAU[dtype], f"{A.name} {dtype} {kw}")


def ragged(n, m, seed, maxlen=40, long_rows=()):
    rng = np.random.default_rng(seed)
    L_ = rng.integers(0, maxlen, n)
    for r, l in long_rows:
        L_[r] = l
    return synth.random_csr(n, m, L_, seed=seed)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("G", [1, 3, 8, 32, 33, 64, 128, 256])
def test_layout_bit_exact_and_spmv_ragged(dtype, G):
    A = ragged(1000, 700, seed=G, long_rows=[(5, 650), (517, 300)])  # tail group partial
    M = to_gpu_matrix(A, dtype, G)
    check_layout(M, A, dtype, G)
    x = synth.uniform_vector(A.n_cols, seed=1)
    for kw in variants(M):
        check_spmv(M, A, dtype, x, **kw)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_small_laplacian_int32_rowptr(dtype):
    A = synth.workload_small_laplacian()
    M = to_gpu_matrix(A, dtype, 32, rowptr_i32=True)
    check_layout(M, A, dtype, 32)
    x = synth.uniform_vector(A.n_cols, seed=0)
    for kw in variants(M):
        check_spmv(M, A, dtype, x, **kw)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_long_rows_and_rectangular(dtype):
    # one row of 10,000 in a group of short rows, several long rows in one
    # warp, a completely empty warp, and n_cols != n_rows
    rng = np.random.default_rng(7)
    n, m = 5000, 12000
    L_ = rng.integers(0, 6, n)
    L_[100] = 10000
    L_[200:204] = [3000, 2500, 40, 9000]
    L_[4000:4032] = 0
    A = synth.random_csr(n, m, L_, seed=7)
    M = to_gpu_matrix(A, dtype, 32)
    check_layout(M, A, dtype, 32)
    x = synth.uniform_vector(m, seed=3)
    for kw in variants(M):
        check_spmv(M, A, dtype, x, **kw)


def test_padding_never_multiplied_nan_canary():
    # padding carries column 0; x[0] = NaN must not reach rows that do not
    # reference column 0
    rng = np.random.default_rng(11)
    A = synth.random_csr(300, 50, rng.integers(0, 20, 300), seed=11)
    keep = A.col != 0
    rows = np.repeat(np.arange(300), A.row_lengths())[keep]
    rowptr = np.zeros(301, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    B = synth.CSRMatrix(300, 50, rowptr, A.col[keep], A.val[keep], "no_col0")
    x = synth.uniform_vector(50, seed=2)
    x[0] = np.nan
    for dtype in ("f32", "f64"):
        M = to_gpu_matrix(B, dtype, 32)
        assert M.n_stored > M.nnz                  # there is padding
        xd = torch.from_numpy(x.astype(NP[dtype])).cuda()
        for kw in variants(M):
            assert torch.isfinite(M.spmv(xd, **kw)).all(), kw


def test_empty_cases():
    for n, m in [(0, 0), (0, 5), (7, 0), (64, 64)]:
        A = synth.random_csr(n, m, np.zeros(n, np.int64))
        M = to_gpu_matrix(A, "f32", 32)
        assert M.n_stored == 0 and M.nnz == 0
        y = M.spmv(torch.zeros(m, dtype=torch.float32, device="cuda"))
        assert y.shape == (n,) and (y == 0).all()


def test_error_codes_from_validation():
    A = ragged(100, 50, seed=1)
    col = A.col.copy()
    col[17] = 50                                    # out of range
    with pytest.raises(L.RgCSRError) as e:
        RgCSRMatrix.from_csr(A.rowptr, col, A.val, 50, dtype=torch.float32)
    assert e.value.status == L.RGCSR_ERR_COL_OOB
    rp = A.rowptr.copy()
    rp[10], rp[11] = rp[11], rp[10] - 1             # decreasing
    with pytest.raises(L.RgCSRError) as e:
        RgCSRMatrix.from_csr(rp, A.col, A.val, 50, dtype=torch.float32)
    assert e.value.status == L.RGCSR_ERR_BAD_ROWPTR
    rp = A.rowptr.copy()
    rp[-1] -= 1                                     # row_ptr[n] != nnz
    with pytest.raises(L.RgCSRError) as e:
        RgCSRMatrix.from_csr(rp, A.col, A.val, 50, dtype=torch.float32)
    assert e.value.status == L.RGCSR_ERR_BAD_ROWPTR


def test_identity_diagonal_permutation_exact():
    n = 4099
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, n)
    d = rng.uniform(-2, 2, n)
    perm = rng.permutation(n).astype(np.int32)
    rp = np.arange(n + 1)
    for dtype in ("f32", "f64"):
        xd = torch.from_numpy(x.astype(NP[dtype])).cuda()
        M = RgCSRMatrix.from_csr(rp, perm, np.ones(n), n, dtype=TT[dtype])
        assert np.array_equal(M.spmv(xd).cpu().numpy(), x.astype(NP[dtype])[perm])
        M = RgCSRMatrix.from_csr(rp, np.arange(n, dtype=np.int32), d, n, dtype=TT[dtype])
        assert np.array_equal(M.spmv(xd).cpu().numpy(), d.astype(NP[dtype]) * x.astype(NP[dtype]))


def test_host_entry_point_matches_device():
    A = ragged(3000, 3000, seed=5)
    M = to_gpu_matrix(A, "f32", 32)
    x = synth.uniform_vector(3000, seed=4).astype(np.float32)
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty(3000, dtype=torch.float32).pin_memory()
    xd = torch.empty(3000, dtype=torch.float32, device="cuda")
    yd = torch.empty(3000, dtype=torch.float32, device="cuda")
    M.spmv_host(xh, yh, xd, yd)
    torch.cuda.synchronize()
    assert torch.equal(yh, M.spmv(torch.from_numpy(x).cuda()).cpu())


# ---------------------------------------------------------------------------
# full-size workloads, group size 32 and the default kernel (as benchmarked)
# ---------------------------------------------------------------------------
FULL = {"a": synth.workload_a, "b": synth.workload_b, "c": synth.workload_c}


@pytest.mark.parametrize("name", ["a", "b", "c"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_full_size_spmv(name, dtype):
    A = FULL[name]()
    M = to_gpu_matrix(A, dtype, 32, slot_map=False)
    rl, gp = oracle_sizes(A, 32)
    assert np.array_equal(M.group_ptr.cpu().numpy(), gp)
    assert np.array_equal(M.row_lengths.cpu().numpy(), rl)
    sample_groups_bit_exact(M, A, dtype, 32, seed=0)
    x = synth.uniform_vector(A.n_cols, seed=0)
    check_spmv(M, A, dtype, x)
    if name != "b":
        check_spmv(M, A, dtype, x, kernel=L.KERNEL_SPLIT)
        check_spmv(M, A, dtype, x, kernel=L.KERNEL_LEAN)
        for v in (1, 2, 4, 5, 6, 7, 8):                     # vector loads (and pipelined)
            check_spmv(M, A, dtype, x, kernel=L.KERNEL_LEAN, variant=v)
        for v in range(7):
            check_spmv(M, A, dtype, x, kernel=L.KERNEL_TMA, variant=v)
    check_spmv(M, A, dtype, x, kernel=L.KERNEL_TMA)
    assert device_status() == 0


_FULL_CACHE = {}


def full_matrix(name):
    if name not in _FULL_CACHE:
        _FULL_CACHE.clear()                      # one full-size matrix in host memory at a time
        _FULL_CACHE[name] = FULL[name]()
    return _FULL_CACHE[name]


def assert_equal_chunked(dev, ref, chunk=1 << 25):
    """Device tensor == host array, element by element (bit patterns for
    floating point), compared in chunks to bound host memory."""
    assert dev.numel() == ref.size
    flat = dev.reshape(-1)
    ui = {8: np.uint64, 4: np.uint32, 2: np.uint16}[ref.itemsize]
    for lo in range(0, ref.size, chunk):
        hi = min(ref.size, lo + chunk)
        got = flat[lo:hi].cpu().numpy()
        if not np.array_equal(got.view(ui), ref[lo:hi].view(ui)):
            bad = lo + int(np.flatnonzero(got.view(ui) != ref[lo:hi].view(ui))[0])
            raise AssertionError(f"first difference at element {bad}")


@pytest.mark.parametrize("name,order", [("a", None), ("c", None), ("b", "descending"), ("b", None)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_full_size_layout_bit_exact(name, order, dtype):
    # every group of the full-size layouts against the oracle's layout
    # builder: row lengths, group pointers, value bits, columns and the slot
    # map (in natural order (b) stores 1,677% artificial zeros at G = 32)
    A = full_matrix(name)
    vals = A.val.astype(NP[dtype])
    perm = oracle.descending_order(A.rowptr) if order else None
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, vals, A.n_cols, group_size=32, dtype=TT[dtype],
                             keep_slot_map=True, row_order=order)
    lay = oracle.rgcsr_layout(A.rowptr, A.col, vals, 32, row_order=perm)
    if order:
        assert_equal_chunked(M.row_perm, perm.astype(np.int32))
    assert M.n_stored == lay.n_stored
    assert_equal_chunked(M.row_lengths, lay.row_lengths)
    assert_equal_chunked(M.group_ptr, lay.group_ptr)
    assert_equal_chunked(M.columns, lay.columns)
    assert_equal_chunked(M.values, lay.values)
    assert_equal_chunked(M.slot_to_csr, lay.slot_to_csr)
    del M, lay
    torch.cuda.empty_cache()


def oracle_sizes(A, G):
    return oracle.rgcsr_sizes(A.rowptr, G)


def sample_groups_bit_exact(M, A, dtype, G, seed, count=300):
    """Oracle layout of sampled groups (each rebuilt from its own rows)."""
    rng = np.random.default_rng(seed)
    n_groups = (A.n_rows + G - 1) // G
    rl = A.row_lengths()
    picks = set(rng.integers(0, n_groups, count).tolist())
    picks.add(n_groups - 1)
    picks.add(int(np.argmax(rl)) // G)
    gp = M.group_ptr.cpu().numpy()
    vals = M.values.cpu().numpy()
    cols = M.columns.cpu().numpy()
    ui = np.uint64 if dtype == "f64" else np.uint32
    for g in sorted(picks):
        r0, r1 = g * G, min(A.n_rows, (g + 1) * G)
        p0, p1 = A.rowptr[r0], A.rowptr[r1]
        sub_rp = A.rowptr[r0:r1 + 1] - p0
        lay = oracle.rgcsr_layout(sub_rp, A.col[p0:p1], A.val[p0:p1].astype(NP[dtype]), G)
        assert lay.n_stored == gp[g + 1] - gp[g]
        assert np.array_equal(cols[gp[g]:gp[g + 1]], lay.columns)
        assert np.array_equal(vals[gp[g]:gp[g + 1]].view(ui), lay.values.view(ui))


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("n", [32, 33, 63, 64, 65, 4095, 100_003])
def test_tma_sizes_and_partial_group(dtype, n):
    # 7-point-like rows with a few longer ones (chunked beyond CAP slot-rows)
    rng = np.random.default_rng(n)
    L_ = rng.integers(5, 8, n)
    L_[rng.integers(0, n, 3)] = rng.integers(20, 60, 3)
    A = synth.random_csr(n, max(n, 64), L_, seed=n)
    M = to_gpu_matrix(A, dtype, 32, slot_map=False)
    x = synth.uniform_vector(A.n_cols, seed=5)
    check_spmv(M, A, dtype, x, kernel=L.KERNEL_TMA)
    for v in (4, 5, 6):                                    # several whole groups per copy
        check_spmv(M, A, dtype, x, kernel=L.KERNEL_TMA, variant=v)
    check_spmv(M, A, dtype, x)
    assert device_status() == 0


@pytest.mark.parametrize("variant", [0, 4])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_tma_bounded_wait_runs_out_then_next_launch_is_correct(dtype, variant):
    # the TMA kernel's waits are bounded: with a limit of one probe the first
    # wait of (nearly) every warp runs out before its bulk copy lands, the
    # kernel records RGCSR_STATUS_TIMEOUT, waits for its own copies in flight
    # and ends; the status read clears the bit, and the next launch with the
    # default limit is correct (the context stays usable)
    A = synth.laplacian_3d(32)
    M = to_gpu_matrix(A, dtype, 32, slot_map=False)
    x = synth.uniform_vector(A.n_cols, seed=3)
    xd = torch.from_numpy(x.astype(NP[dtype])).cuda()
    assert device_status() == 0
    y = torch.full((A.n_rows,), float("nan"), dtype=TT[dtype], device="cuda")
    M.spmv(xd, out=y, kernel=L.KERNEL_TMA, variant=variant, wait_limit=1)
    torch.cuda.synchronize()
    assert device_status() == L.STATUS_TIMEOUT
    assert torch.isnan(y).any()                    # rows of the abandoned groups stay unwritten
    assert device_status() == 0                    # the read cleared the bit
    check_spmv(M, A, dtype, x, kernel=L.KERNEL_TMA, variant=variant)
    assert device_status() == 0
    with pytest.raises(L.RgCSRError):
        M.spmv(xd, out=y, kernel=L.KERNEL_TMA, wait_limit=-1)


# ---------------------------------------------------------------------------
# x staged in shared memory (x-window arm of the read-path study)
# ---------------------------------------------------------------------------
def expected_windows(A, G, perm, x_bytes):
    """The plan's definition restated on the host: per block of 256 stored
    rows, the sorted distinct columns of its entries cut where consecutive
    columns are more than 64 apart; kept if at most 4 ranges of at most
    32 KB of x, with at most 8,192 entries in the block."""
    n = A.n_rows
    rows = np.arange(n) if perm is None else np.asarray(perm)
    out = []
    for b in range((n + 255) // 256):
        cols = [A.col[A.rowptr[r]:A.rowptr[r + 1]] for r in rows[b * 256:(b + 1) * 256]]
        total = sum(c.size for c in cols)
        if total == 0 or total > 8192:
            out.append((0, 0, [], []))
            continue
        u = np.unique(np.concatenate(cols))
        cut = np.flatnonzero(np.diff(u) > 64)
        if cut.size > 3:
            out.append((0, 0, [], []))
            continue
        starts = np.concatenate([[u[0]], u[cut + 1]])
        ends = np.concatenate([u[cut], [u[-1]]]) + 1
        lens = ends - starts
        if lens.sum() > 32768 // x_bytes:
            out.append((0, 0, [], []))
            continue
        out.append((len(starts), int(lens.sum()), starts.tolist(), lens.tolist()))
    return out


def banded(n, half, seed):
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        c = np.arange(max(0, i - half), min(n, i + half + 1))
        rows.append(c.size)
        cols.append(c)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(rows, out=rp[1:])
    return synth.CSRMatrix(n, n, rp, np.concatenate(cols).astype(np.int32), rng.uniform(-1, 1, int(rp[-1])),
                           f"band{half}")


def four_bands(n, seed):
    """Row i holds columns i, i + n/4, i + n/2, i + 3n/4 (mod n): four
    separated ranges per block, five where a block wraps around."""
    rng = np.random.default_rng(seed)
    cols = np.sort((np.arange(n)[:, None] + np.arange(4)[None, :] * (n // 4)) % n, axis=1)
    rp = np.arange(n + 1, dtype=np.int64) * 4
    return synth.CSRMatrix(n, n, rp, cols.reshape(-1).astype(np.int32), rng.uniform(-1, 1, 4 * n), "four_bands")


XWIN_CASES = {
    "four_bands": lambda: four_bands(4000, 3),                  # four ranges (five: not staged)
    "ragged_6k": lambda: ragged(2000, 6000, seed=7, maxlen=20),  # one range of > 4,096: FP32 only
    "laplace3d_32": lambda: synth.laplacian_3d(32),              # three bands per block
    "laplace3d_16": lambda: synth.laplacian_3d(16),              # adjacent planes: one range
    "laplace2d_64": lambda: synth.workload_small_laplacian(),    # one range
    "stencil27_12": lambda: synth.stencil27_random(12),
    "band_13_odd_n": lambda: banded(5003, 13, 1),                # one range; partial last block
    "band_37": lambda: banded(3000, 37, 1),                      # > 8,192 entries per block: not staged
    "ragged_narrow": lambda: ragged(3001, 2000, seed=4),         # random columns, narrow: one range
    "ragged_wide": lambda: ragged(3001, 200000, seed=4, maxlen=20),   # random columns: not staged
    "long_row": lambda: ragged(1000, 900, seed=5, long_rows=[(3, 850)]),
}


@pytest.mark.parametrize("name", sorted(XWIN_CASES))
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("G,order", [(32, None), (7, None), (32, "descending")])
def test_xwindow_plan_and_spmv(name, dtype, G, order):
    A = XWIN_CASES[name]()
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=G, dtype=TT[dtype],
                             row_order=order).plan_x_window()
    perm = None if M.row_perm is None else M.row_perm.cpu().numpy()
    got = M.x_window_records()
    want = expected_windows(A, G, perm, 8 if dtype == "f64" else 4)
    for b, (g_, w_) in enumerate(zip(got, want)):
        assert g_[0] == w_[0] and g_[1] == w_[1], (b, g_, w_)
        assert g_[2][:w_[0]] == w_[2] and g_[3][:w_[0]] == w_[3], (b, g_, w_)
    x = synth.uniform_vector(A.n_cols, seed=2)
    xd = torch.from_numpy(x.astype(NP[dtype])).cuda()
    y = M.spmv_xwindow(xd).cpu().numpy()
    y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, rounded_values(A.val, dtype), rounded_values(x, dtype))
    assert_within_bound(y, y_ref, absy, TAU[dtype], f"{name} xwindow")


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_xwindow_reduced_storage(fmt):
    A = synth.laplacian_3d(32)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=32, dtype=torch.float64)
    Q = M.quantized(fmt).plan_x_window()
    recs = Q.x_window_records()
    assert [r[:2] for r in recs] == [w[:2] for w in expected_windows(A, 32, None, 4)]
    assert all(r[0] == 3 for r in recs[4:-4])     # blocks off the first and last z-planes: three bands
    x = synth.uniform_vector(A.n_cols, seed=3).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    assert torch.equal(Q.spmv_xwindow(xd), Q.spmv(xd, kernel=L.KERNEL_LEAN))   # same order, same sums


def test_texture_cache_overflow():
    # more x buffers than the library keeps texture objects for: the cache
    # is cleared (after a device synchronisation) and products stay right
    A = ragged(500, 400, seed=6)
    M = to_gpu_matrix(A, "f32", 8, slot_map=False)
    for i in range(70):
        x = synth.uniform_vector(A.n_cols, seed=100 + i)
        check_spmv(M, A, "f32", x, kernel=L.KERNEL_SPLIT, x_load=L.XLOAD_TEX)


def test_x_load_needs_a_scalar_kernel():
    A = synth.workload_small_laplacian()
    M = to_gpu_matrix(A, "f32", 32, slot_map=False)
    xd = torch.zeros(A.n_cols, dtype=torch.float32, device="cuda")
    for kw in (dict(x_load=L.XLOAD_TEX), dict(kernel=L.KERNEL_TMA, x_load=L.XLOAD_PLAIN),
               dict(kernel=L.KERNEL_LEAN, variant=1, x_load=L.XLOAD_TEX), dict(kernel=L.KERNEL_SPLIT, x_load=3)):
        with pytest.raises(L.RgCSRError):
            M.spmv(xd, **kw)


# ---------------------------------------------------------------------------
# long-row segment schedule
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("G,T,S", [(32, 64, 256), (1, 16, 32), (8, 0, 64), (33, 5, 7), (32, 100000, 256)])
def test_long_row_segments(dtype, G, T, S):
    rng = np.random.default_rng(G + T + S)
    n, m = 3000, 20000
    L_ = rng.integers(0, 10, n)
    L_[[1, 2, 100, 2999]] = [12000, 700, 65, 3000]
    A = synth.random_csr(n, m, L_, seed=5)
    M = to_gpu_matrix(A, dtype, G, slot_map=False).split_long_rows(threshold=T, segment=S)
    expected = int(sum((l - T + S - 1) // S for l in L_ if l > T))
    assert M.n_long_segments == expected
    check_spmv(M, A, dtype, synth.uniform_vector(m, seed=8))


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_long_row_segments_repeat_bitwise(dtype):
    # the last segment of a row to finish adds its partials in a fixed order:
    # repeated products on one schedule agree bit for bit, and every arrival
    # counter is back at zero after each product
    rng = np.random.default_rng(11)
    n, m = 4000, 50000
    L_ = rng.integers(0, 12, n)
    L_[[0, 7, 1234, 3999]] = [40000, 2048, 33 * 64 + 1, 700]
    A = synth.random_csr(n, m, L_, seed=12)
    M = to_gpu_matrix(A, dtype, 4, slot_map=False).split_long_rows(threshold=16, segment=64)
    x = torch.from_numpy(synth.uniform_vector(m, seed=13)).cuda().to(M.x_dtype)
    arrivals = M._long[1]["arrivals"]
    first = M.spmv(x)
    assert int(arrivals.abs().sum()) == 0
    for _ in range(4):
        y = M.spmv(x)
        assert torch.equal(y, first)
        assert int(arrivals.abs().sum()) == 0
    check_spmv(M, A, dtype, synth.uniform_vector(m, seed=13))


def test_long_row_segments_quantized():
    A = synth.power_law(20000, seed=4)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=8, dtype=torch.float64)
    Q = M.quantized("bf16").split_long_rows(threshold=32, segment=128)
    x = synth.uniform_vector(A.n_cols, seed=1).astype(np.float32)
    y = Q.spmv(torch.from_numpy(x).cuda()).cpu().numpy()
    y_plain = Q.spmv(torch.from_numpy(x).cuda(), kernel=L.KERNEL_SPLIT).cpu().numpy()
    q, sc = oracle.quantize_rows(A.rowptr, A.val, oracle.BF16)
    deq = oracle.dequantized_values(A.rowptr, q, sc, oracle.BF16)
    y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, deq, x.astype(np.float64))
    assert_within_bound(y, y_ref, absy, 2e-6, "segments bf16")
    assert_within_bound(y_plain, y_ref, absy, 2e-6, "split bf16")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("G", [1, 8, 32])
def test_long_row_segments_full_size_b(dtype, G):
    A = synth.workload_b()
    M = to_gpu_matrix(A, dtype, G, slot_map=False).split_long_rows(threshold=64, segment=256)
    check_spmv(M, A, dtype, synth.uniform_vector(A.n_cols, seed=0))


def test_unknown_kernel_variants_rejected():
    A = ragged(300, 200, seed=2)
    M = to_gpu_matrix(A, "f32", 32)
    x = torch.zeros(A.n_cols, dtype=torch.float32, device="cuda")
    for kw in (dict(kernel=L.KERNEL_LEAN, variant=3), dict(kernel=L.KERNEL_LEAN, variant=10),
               dict(kernel=L.KERNEL_LEAN, variant=9),                   # BF16/FP16 storage only
               dict(kernel=L.KERNEL_TMA, variant=7),
               dict(kernel=L.KERNEL_LEAN, variant=-1)):
        with pytest.raises(L.RgCSRError) as e:
            M.spmv(x, **kw)
        assert e.value.status == L.RGCSR_ERR_INVALID_ARG


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("G", [1, 5, 32])
def test_sliced_ellpack_comparator(dtype, G):
    # the comparator runs all K_g slots of every row: equal to the oracle's
    # sliced ELLPACK product, NaN wherever x[0] = NaN meets padding, and
    # equal to the CSR product when x is finite
    rng = np.random.default_rng(G)
    A = synth.random_csr(700, 90, rng.integers(0, 25, 700), seed=G)
    M = to_gpu_matrix(A, dtype, G)
    lay = oracle.rgcsr_layout(A.rowptr, A.col, A.val.astype(NP[dtype]), G)
    x = synth.uniform_vector(A.n_cols, seed=4)
    check_spmv(M, A, dtype, x, kernel=L.KERNEL_SELL)
    x[0] = np.nan
    y = M.spmv(torch.from_numpy(x.astype(NP[dtype])).cuda(), kernel=L.KERNEL_SELL).cpu().numpy()
    y_sell = oracle.sliced_ell_spmv(lay, rounded_values(x, dtype))
    assert np.array_equal(np.isnan(y), np.isnan(y_sell))
    ok = ~np.isnan(y_sell)
    _, absy = oracle.csr_spmv(A.rowptr, A.col, rounded_values(A.val, dtype), np.nan_to_num(rounded_values(x, dtype)))
    assert (np.abs(y[ok] - y_sell[ok]) <= TAU[dtype] * absy[ok]).all()
    if G > 1:
        assert np.isnan(y_sell).any() and not np.isnan(M.spmv(torch.from_numpy(x.astype(NP[dtype])).cuda()).cpu().numpy()).all()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("G,order", [(32, None), (32, "descending"), (8, None), (1, None)])
def test_layout_with_big_groups(dtype, G, order):
    # groups whose slab exceeds the per-group scatter's limit (rows of 300 to
    # 9000 slots) are written one warp per row: still bit-exact
    rng = np.random.default_rng(G)
    n, m = 3000, 10000
    L_ = rng.integers(0, 20, n)
    L_[[5, 6, 40, 1000, 2999]] = [9000, 300, 4000, 260, 7000]
    A = synth.random_csr(n, m, L_, seed=G)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=G, dtype=TT[dtype],
                             keep_slot_map=True, row_order=order)
    perm = oracle.descending_order(A.rowptr) if order else None
    lay = oracle.rgcsr_layout(A.rowptr, A.col, A.val.astype(NP[dtype]), G, row_order=perm)
    ui = np.uint64 if dtype == "f64" else np.uint32
    assert np.array_equal(M.values.cpu().numpy().view(ui), lay.values.view(ui))
    assert np.array_equal(M.columns.cpu().numpy(), lay.columns)
    assert np.array_equal(M.slot_to_csr.cpu().numpy(), lay.slot_to_csr)
    check_spmv(M, A, dtype, synth.uniform_vector(m, seed=1))


@pytest.mark.parametrize("name", list(synth.TABLE6_ROWS))
def test_table6_standins(name):
    # the four matrix shapes of Sec. 4.4.2 (Table 6), FP64 as in the paper:
    # layout at G = 128 (the paper's setting) against the oracle, and the SpMV
    # of the paper's kernel at G = 128, the default at G = 32, the warp split,
    # descending order with group tiles, and HYB, within tau |A||x|
    A = synth.table6_standin(name)
    x = synth.uniform_vector(A.n_cols, seed=11)
    M = to_gpu_matrix(A, "f64", 128, slot_map=False)
    rl, gp = oracle_sizes(A, 128)
    assert np.array_equal(M.group_ptr.cpu().numpy(), gp) and np.array_equal(M.row_lengths.cpu().numpy(), rl)
    check_spmv(M, A, "f64", x, kernel=L.KERNEL_PAPER)
    M32 = to_gpu_matrix(A, "f64", 32, slot_map=False)
    check_spmv(M32, A, "f64", x)
    check_spmv(M32, A, "f64", x, kernel=L.KERNEL_SPLIT)
    D = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=32, dtype=torch.float64,
                             row_order="descending").tile_groups(64)
    check_spmv(D, A, "f64", x)
    H = HybMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, dtype=torch.float64)
    check_spmv(H, A, "f64", x)
    assert device_status() == 0


def test_gather_probe_counts_and_writes_nothing():
    from paper_1012_2270_gb300.rgcsr import gather_probe, _FMA_SINKS
    x = torch.ones(1 << 12, dtype=torch.float64, device="cuda")
    n = gather_probe(x, iters=2)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert n == sms * 1024 * 4 * 2
    torch.cuda.synchronize()
    assert float(_FMA_SINKS[x.device]) == 0.0
    with pytest.raises(L.RgCSRError):
        gather_probe(torch.ones(1000, dtype=torch.float64, device="cuda"))      # not a power of two
