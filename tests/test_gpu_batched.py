"""GPU parity of the batched SpMV: every member of an uneven batch (banded,
stencil and power-law members, mixed group sizes) against the oracle's CSR
SpMV, equality with per-member SpMV, CUDA-graph replay, and the autotuner
returning a configuration that computes the right product."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TAU, assert_within_bound, rounded_values
from paper_1012_2270_gb300 import synth
from paper_1012_2270_gb300 import autotune
from paper_1012_2270_gb300.batched import BatchedRgCSR, BlockDiagonalBatch
from paper_1012_2270_gb300.rgcsr import RgCSRMatrix

pytestmark = pytest.mark.gpu

NP = {"f32": np.float32, "f64": np.float64}
TT = {"f32": torch.float32, "f64": torch.float64}


def small_batch(count=48):
    return [synth.batch_member(i, n_min=200, n_max=20000) for i in range(count)]


def check_batch(mats, Bt, dtype, x_cat, y_cat):
    for i, A in enumerate(mats):
        xs, ys = Bt.member_slices(i)
        x = x_cat[xs].double().cpu().numpy()
        y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, rounded_values(A.val, dtype), x)
        assert_within_bound(y_cat[ys].cpu().numpy(), y_ref, absy, TAU[dtype], f"member {i} {A.name}")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("groups", ["model", 32, 8])
def test_batched_members_match_oracle(dtype, groups):
    mats = small_batch()
    Bt = BatchedRgCSR.from_csr_list(mats, dtype=TT[dtype], group_sizes=groups)
    x_cat = torch.from_numpy(synth.uniform_vector(Bt.n_cols_total, seed=3).astype(NP[dtype])).cuda()
    y_cat = Bt.spmv(x_cat)
    check_batch(mats, Bt, dtype, x_cat, y_cat)


def test_batched_equals_per_member_and_graph_replay():
    mats = small_batch(30)
    Bt = BatchedRgCSR.from_csr_list(mats, dtype=torch.float32)
    x_cat = torch.from_numpy(synth.uniform_vector(Bt.n_cols_total, seed=4).astype(np.float32)).cuda()
    y_cat = torch.full((Bt.n_rows_total,), float("nan"), device="cuda")
    g = Bt.capture(x_cat, y_cat, repeats=3)
    y_cat.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    y_direct = Bt.spmv(x_cat)
    assert torch.equal(y_cat, y_direct)
    for i, A in enumerate(mats):
        xs, ys = Bt.member_slices(i)
        M = RgCSRMatrix.from_csr(A.rowptr, A.col, A.val, A.n_cols, group_size=Bt.group_sizes[i],
                                 dtype=torch.float32)
        y = M.spmv(x_cat[xs].contiguous(), kernel=2)       # the same split algorithm
        assert torch.equal(y, y_direct[ys]), i


def test_batched_with_empty_members():
    mats = [synth.random_csr(0, 5, np.zeros(0, np.int64)), synth.laplacian_2d(9),
            synth.random_csr(40, 3, np.zeros(40, np.int64)), synth.power_law(3000, seed=2)]
    Bt = BatchedRgCSR.from_csr_list(mats, dtype=torch.float64)
    x_cat = torch.from_numpy(synth.uniform_vector(Bt.n_cols_total, seed=5)).cuda()
    y_cat = Bt.spmv(x_cat)
    check_batch(mats, Bt, "f64", x_cat, y_cat)


def test_autotune_returns_a_correct_configuration(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE_PATH", str(tmp_path / "tune.json"))
    A = synth.power_law(50000, seed=3)
    best = autotune.tune(A.rowptr, A.col, A.val.astype(np.float32), A.n_cols, dtype=torch.float32, reps=3)
    assert best["us"] > 0
    M, kw = autotune.build(A.rowptr, A.col, A.val.astype(np.float32), A.n_cols, best, torch.float32)
    x = synth.uniform_vector(A.n_cols, seed=0).astype(np.float32)
    y = M.spmv(torch.from_numpy(x).cuda(), **kw).cpu().numpy()
    y_ref, absy = oracle.csr_spmv(A.rowptr, A.col, rounded_values(A.val, "f32"), x.astype(np.float64))
    assert_within_bound(y, y_ref, absy, TAU["f32"], "autotuned")
    # cached on the second call
    again = autotune.tune(A.rowptr, A.col, A.val.astype(np.float32), A.n_cols, dtype=torch.float32, reps=3)
    assert again == best
    hb = autotune.tune_hyb_width(A.rowptr, A.col, A.val.astype(np.float32), A.n_cols, reps=3)
    assert hb["ell_width"] >= 0


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("order,tile", [("descending", 64), ("descending", 8), (None, 16), (None, None)])
def test_block_diagonal_batch(dtype, order, tile):
    mats = small_batch(36)
    mats.insert(5, synth.random_csr(0, 7, np.zeros(0, np.int64)))          # an empty member
    Bd = BlockDiagonalBatch.from_csr_list(mats, dtype=TT[dtype], row_order=order, tile=tile)
    x_cat = torch.from_numpy(synth.uniform_vector(Bd.n_cols_total, seed=6).astype(NP[dtype])).cuda()
    y_cat = Bd.spmv(x_cat)
    check_batch(mats, Bd, dtype, x_cat, y_cat)
    y2 = torch.full_like(y_cat, float("nan"))
    g = Bd.capture(x_cat, y2, repeats=2)
    y2.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y2, y_cat)                                           # deterministic, replayable


@pytest.mark.parametrize("tile,variant", [(128, 7), (256, 7)])
def test_block_diagonal_full_batch_sampled(tile, variant):
    # the benchmark's 512-member batch in the block-diagonal configurations
    # it times fastest: every member's rows checked against the oracle
    mats = synth.workload_batch(512)
    Bd = BlockDiagonalBatch.from_csr_list(mats, dtype=torch.float32, tile=tile, variant=variant)
    x_cat = torch.from_numpy(synth.uniform_vector(Bd.n_cols_total, seed=9).astype(np.float32)).cuda()
    y_cat = Bd.spmv(x_cat)
    check_batch(mats, Bd, "f32", x_cat, y_cat)
