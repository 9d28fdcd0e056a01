"""GPU parity of the group-tile schedule (one warp per tile of at most C
slot-rows of a row group, long groups cut into several tiles whose
partials the last-arriving tile adds in order) against the CPU oracle:
schedule sizes from the oracle's group sizes, y within tau*|A||x| for
natural and descending row order, bit-identical repeated launches (the
per-group arrival counters reset themselves), reduced-precision storage,
the host entry point, and argument errors."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from helpers import TAU, assert_within_bound, rounded_values
from paper_1012_2270_gb300 import synth
from paper_1012_2270_gb300 import _lib as L
from paper_1012_2270_gb300.rgcsr import RgCSRMatrix, _ptr, _stream_ptr

pytestmark = pytest.mark.gpu

NP = {"f32": np.float32, "f64": np.float64}
TT = {"f32": torch.float32, "f64": torch.float64}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1012_2270_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def ragged(n, m, seed):
    rng = np.random.default_rng(seed)
    lengths = rng.integers(0, 12, n)
    lengths[rng.integers(0, n, 4)] = [3000, 700, 129, 64]
    return synth.random_csr(n, m, lengths, seed=seed)


def expected_schedule(A, G, C, perm=None):
    """(extra tiles, split groups) from the oracle's group pointers."""
    lengths = np.diff(A.rowptr)
    if perm is not None:
        lengths = lengths[perm]
    _, gp = oracle.rgcsr_sizes(np.concatenate([[0], np.cumsum(lengths)]), G)
    n = lengths.size
    extra = split = 0
    for g in range(gp.size - 1):
        R = min(G, n - g * G)
        K = (gp[g + 1] - gp[g]) // R
        tasks = -(-K // C) if K > C else 1
        extra += tasks - 1
        split += tasks > 1
    return extra, split


def check(M, A, dtype, x):
    xd = torch.from_numpy(x.astype(NP[dtype])).cuda()
    y1 = M.spmv(xd).cpu().numpy()
    y2 = M.spmv(xd).cpu().numpy()
    assert np.array_equal(y1.view(np.uint8), y2.view(np.uint8)), "repeated launch differs"
    y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, rounded_values(A.val, dtype), rounded_values(x, dtype))
    assert_within_bound(y1, y_ref, absy, TAU[dtype], f"tiles {dtype}")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("G", [1, 7, 32])
@pytest.mark.parametrize("C", [1, 3, 16, 64, 1 << 20])
@pytest.mark.parametrize("order", [None, "descending"])
def test_tiles_ragged(dtype, G, C, order):
    A = ragged(2001, 4000, seed=G * 7 + C % 97)          # partial last group for G = 7, 32
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=G,
                             dtype=TT[dtype], row_order=order).tile_groups(C)
    perm = oracle.descending_order(A.rowptr) if order else None
    extra, split = expected_schedule(A, G, C, perm)
    T = M._tiles[0]
    assert (T.n_extra, T.n_split, T.n_partials) == (extra, split, extra + split)
    check(M, A, dtype, synth.uniform_vector(A.n_cols, seed=3))


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_tiles_quantized(fmt):
    A = synth.power_law(30_000, seed=9)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=32, dtype=torch.float64,
                             row_order="descending")
    Q = M.quantized(fmt).tile_groups(32)
    code = oracle.BF16 if fmt == "bf16" else oracle.F16
    q, sc = oracle.quantize_rows(A.rowptr, A.val, code)
    deq = oracle.dequantized_values(A.rowptr, q, sc, code)
    x = synth.uniform_vector(A.n_cols, seed=1).astype(np.float32)
    y = Q.spmv(torch.from_numpy(x).cuda()).cpu().numpy()
    y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, deq, x.astype(np.float64))
    assert_within_bound(y, y_ref, absy, 2e-6, f"tiles {fmt}")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_tiles_host_path(dtype):
    A = ragged(5000, 6000, seed=4)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=32,
                             dtype=TT[dtype], row_order="descending").tile_groups(16)
    x = synth.uniform_vector(A.n_cols, seed=4).astype(NP[dtype])
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty(A.n_rows, dtype=TT[dtype]).pin_memory()
    M.spmv_host(xh, yh, torch.empty_like(xh, device="cuda"), torch.empty_like(yh, device="cuda"))
    torch.cuda.synchronize()
    y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, rounded_values(A.val, dtype), x.astype(np.float64))
    assert_within_bound(yh.numpy(), y_ref, absy, TAU[dtype], "tiles host path")


def test_tiles_errors_and_empty():
    A = ragged(300, 4000, seed=5)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=64)
    with pytest.raises(L.RgCSRError) as e:
        M.tile_groups(16)                                   # G > 32
    assert e.value.status == L.RGCSR_ERR_INVALID_ARG
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=32)
    with pytest.raises(L.RgCSRError):
        M.tile_groups(0)
    M.tile_groups(8)
    T = M._tiles[0]
    x = torch.zeros(A.n_cols, dtype=torch.float64, device="cuda")
    y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
    bad = L.Tiles.from_buffer_copy(T)
    bad.n_groups = T.n_groups + 1                           # schedule of another matrix
    st = L.lib().rgcsr_spmv_tiles(ctypes.byref(M.s), ctypes.byref(bad), _ptr(x), _ptr(y), _stream_ptr())
    assert st == L.RGCSR_ERR_INVALID_ARG
    E = RgCSRMatrix.from_csr(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), 5, group_size=32)
    E.tile_groups(4)
    assert E.spmv(torch.zeros(5, dtype=torch.float64, device="cuda")).numel() == 0


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_tiles_full_size_b_descending(dtype):
    # every tile shape the benchmark's tuner may pick for the power-law matrix
    A = synth.workload_b()
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=32,
                             dtype=TT[dtype], row_order="descending")
    x = synth.uniform_vector(A.n_cols, seed=0)
    for C in (32, 64, 128):
        for v in range(8):
            M._tiles = None
            M.tile_groups(C, variant=v)
            check(M, A, dtype, x)


@pytest.mark.parametrize("name", ["a", "c"])
def test_tiles_full_size_stencils(name):
    A = {"a": synth.workload_a, "c": synth.workload_c}[name]()
    for dtype in ("f32", "f64"):
        M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=32,
                                 dtype=TT[dtype]).tile_groups(64)
        assert M.n_extra_tiles == 0
        check(M, A, dtype, synth.uniform_vector(A.n_cols, seed=0))


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("C", [3, 64])
def test_tiles_variants(dtype, variant, C):
    A = ragged(3001, 4000, seed=variant * 10 + C)
    M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=32,
                             dtype=TT[dtype], row_order="descending").tile_groups(C, variant=variant)
    check(M, A, dtype, synth.uniform_vector(A.n_cols, seed=6))
    bad = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(NP[dtype]), A.n_cols, group_size=32,
                               dtype=TT[dtype]).tile_groups(C, variant=8)
    with pytest.raises(L.RgCSRError):
        bad.spmv(torch.zeros(A.n_cols, dtype=TT[dtype], device="cuda"))
