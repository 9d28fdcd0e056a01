"""The library's structural checks of an RgCSR matrix (rgcsr_check_matrix)
and its checks mode, in which every product checks its matrix first.

Valid matrices of every kind pass.  Each corruption is planted on the host
side of the test (a torch write into one array of a freshly converted
matrix) and must be reported with its check and the lowest failing index.
Only the check kernel ever reads a corrupt matrix: it stays inside the
sizes the descriptor declares.  In checks mode a product on a corrupt
matrix must refuse before any kernel runs (its output stays untouched);
the one corruption used there is a column just past n_cols, with x
allocated longer than n_cols, so even a product that ran would stay inside
x's memory."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1012_2270_gb300 import _lib as L
from paper_1012_2270_gb300 import synth
from paper_1012_2270_gb300.rgcsr import RgCSRMatrix, get_status, set_checks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1012_2270_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def ragged(n=300, m=280, seed=3):
    rng = np.random.default_rng(seed)
    lengths = rng.integers(0, 12, size=n)
    lengths[::17] = 0                       # empty rows
    lengths[5] = 40                         # one long row
    return synth.random_csr(n, m, lengths, seed=seed)


def convert(A, G=32, dtype=torch.float32, order=None, slot_map=True):
    np_t = np.float64 if dtype == torch.float64 else np.float32
    return RgCSRMatrix.from_csr(A.rowptr, A.col, A.val.astype(np_t), A.n_cols, group_size=G, dtype=dtype,
                                keep_slot_map=slot_map, row_order=order)


def slots(M):
    """Host lists of valid and padding slots as (slot, stored row)."""
    gp = M.group_ptr.cpu().numpy()
    rl = M.row_lengths.cpu().numpy()
    G, n = M.s.group_size, M.s.n_rows
    valid, pad = [], []
    for g in range(M.s.n_groups):
        R = min(G, n - g * G)
        K = (gp[g + 1] - gp[g]) // R
        for j in range(K):
            for t in range(R):
                (valid if j < rl[g * G + t] else pad).append((int(gp[g] + j * R + t), g * G + t))
    return valid, pad


@pytest.mark.parametrize("G", [1, 3, 32, 33])
@pytest.mark.parametrize("order", [None, "descending"])
def test_valid_matrices_pass(G, order):
    M = convert(ragged(), G=G, order=order)
    rep = M.check()
    assert rep == {"ok": True, "flags": [], "group": -1, "row": -1, "slot": -1}
    Q = M.quantized("bf16")
    assert Q.check()["ok"]
    D = convert(ragged(), G=G, dtype=torch.float64, order=order, slot_map=False)
    assert D.check()["ok"]


def test_workload_sizes_pass():
    for A in (synth.workload_small_laplacian(), synth.stencil27_random(24)):
        assert convert(A).check()["ok"]


def test_empty_matrix_passes():
    A = synth.random_csr(0, 5, np.zeros(0, dtype=np.int64))
    assert convert(A).check()["ok"]


def _corrupt(kind):
    """A fresh matrix with one planted corruption; returns (M, expected
    flags, expected report entries)."""
    A = ragged()
    M = convert(A, order="descending" if kind.startswith("perm") else None)
    valid, pad = slots(M)
    n, m = M.s.n_rows, M.s.n_cols
    rl = M.row_lengths.cpu().numpy()
    if kind == "column_high":
        s = valid[len(valid) // 2][0]
        M.columns[s] = m + 3
        return M, {"column"}, {"slot": s}
    if kind == "column_negative":
        s = valid[7][0]
        M.columns[s] = -1
        return M, {"column"}, {"slot": s}
    if kind == "padding_value":
        s = pad[len(pad) // 3][0]
        M.values[s] = 1.0
        return M, {"padding"}, {"slot": s}
    if kind == "padding_column":
        s = pad[-1][0]
        M.columns[s] = 5
        return M, {"padding"}, {"slot": s}
    if kind == "length_sum":
        # a row shorter than its group's longest gains one slot: the slab
        # sizes still hold, the lengths no longer sum to nnz
        G = M.s.group_size
        r = next(r for r in range(n) if 0 < rl[r] < rl[(r // G) * G:(r // G + 1) * G].max())
        M.row_lengths[r] = int(rl[r]) + 1          # its first padding slot turns valid: slot map -1
        return M, {"row_lengths", "slot_map"}, {}
    if kind == "length_negative":
        r = int(np.argmax(rl == 0))
        M.row_lengths[r] = -1
        return M, {"row_lengths"}, {"row": r}
    if kind == "length_over_max":
        r = 5
        M.row_lengths[r] = int(M.s.max_row_len) + 1
        return M, {"row_lengths", "group_ptr"}, {"row": r, "group": r // M.s.group_size}
    if kind == "group_ptr":
        g = M.s.n_groups // 2
        M.group_ptr[g] += 1
        return M, {"group_ptr"}, {"group": g - 1}
    if kind == "group_ptr_end":
        M.group_ptr[M.s.n_groups] -= 1
        return M, {"group_ptr"}, {"group": M.s.n_groups - 1}
    if kind == "perm_range":
        r = n // 2
        M.row_perm[r] = n
        return M, {"perm"}, {"row": r}
    if kind == "perm_duplicate":
        M.row_perm[10] = M.row_perm[20].item()
        return M, {"perm"}, {}
    if kind == "slot_map":
        s = valid[3][0]
        M.slot_to_csr[s] = M.s.nnz
        return M, {"slot_map"}, {"slot": s}
    if kind == "slot_map_padding":
        s = pad[0][0]
        M.slot_to_csr[s] = 0
        return M, {"slot_map"}, {"slot": s}
    if kind == "scale":
        Q = M.quantized("bf16")
        Q.row_scale[9] = float("nan")
        return Q, {"scale"}, {"row": 9}
    raise ValueError(kind)


KINDS = ["column_high", "column_negative", "padding_value", "padding_column", "length_sum", "length_negative",
         "length_over_max", "group_ptr", "group_ptr_end", "perm_range", "perm_duplicate", "slot_map",
         "slot_map_padding", "scale"]


@pytest.mark.parametrize("kind", KINDS)
def test_corruption_is_reported(kind):
    M, flags, where = _corrupt(kind)
    rep = M.check()
    assert not rep["ok"]
    if kind == "group_ptr":
        # the two groups' slots are read with shifted coordinates as well
        assert "group_ptr" in rep["flags"] and set(rep["flags"]) <= {"group_ptr", "padding", "slot_map"}
    else:
        assert set(rep["flags"]) == flags, rep
    for k, v in where.items():
        assert rep[k] == v, (rep, where)


def test_descriptor_errors():
    M = convert(ragged())
    rep = L.CheckReport()
    st = L.lib().rgcsr_check_matrix(None, ctypes.byref(rep), None)
    assert st == L.RGCSR_ERR_INVALID_ARG
    assert L.lib().rgcsr_check_matrix(ctypes.byref(M.s), None, None) == L.RGCSR_ERR_INVALID_ARG
    bad = L.Matrix.from_buffer_copy(M.s)
    bad.n_groups += 1
    assert L.lib().rgcsr_check_matrix(ctypes.byref(bad), ctypes.byref(rep), None) == L.RGCSR_ERR_INVALID_ARG


def test_checks_mode_refuses_a_corrupt_matrix():
    A = ragged()
    M = convert(A)
    good = convert(A)
    valid, _ = slots(M)
    m = M.s.n_cols
    x_mem = torch.rand(m + 64, device="cuda")      # longer than n_cols: see the module docstring
    x = x_mem[:m]
    y_good = good.spmv(x)
    X = torch.rand(m + 64, 4, device="cuda")[:m]          # a contiguous view of a longer buffer
    M.columns[valid[11][0]] = m + 3
    get_status()                                    # clear
    prev = set_checks(True)
    try:
        y = torch.full((M.s.n_rows,), 7.0, device="cuda")
        with pytest.raises(L.RgCSRError) as e:
            M.spmv(x, out=y)
        assert e.value.status == L.RGCSR_ERR_CORRUPT
        torch.cuda.synchronize()
        assert torch.all(y == 7.0)                  # nothing was launched
        assert get_status() & L.STATUS_CORRUPT
        assert get_status() == 0                    # the read cleared it
        Y = torch.full((M.s.n_rows, 4), 7.0, device="cuda")
        with pytest.raises(L.RgCSRError):
            M.spmm(X, out=Y)
        torch.cuda.synchronize()
        assert torch.all(Y == 7.0)
        M.tile_groups(64)
        with pytest.raises(L.RgCSRError):
            M.spmv(x, out=y)
        torch.cuda.synchronize()
        assert torch.all(y == 7.0)
        get_status()
        # a valid matrix runs as before, with nothing raised
        assert torch.equal(good.spmv(x), y_good)
        good.tile_groups(64)
        torch.testing.assert_close(good.spmv(x), y_good, rtol=1e-6, atol=1e-6)
        assert get_status() == 0
    finally:
        set_checks(prev)
