"""The benchmark's multi-process path on CPU (world_size 2, gloo): N
replicas, each timing its own SpMVs, report the whole-job throughput over
the slowest replica's time; the reference arm prints from rank 0 only.  The
SpMV itself does not shard (replicas only), so no data-path collective is
tested here."""
import contextlib
import io
import json
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r timed (1 + r) ms for the step loop and (10 - r) ms end to end
    got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 3.0])
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(got, f)
    dist.destroy_process_group()


def test_max_over_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    results = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert results[0] == results[1] == [2.0, 10.0, 3.0]


def test_single_process_and_whole_job_value():
    import bench
    assert bench.max_over_ranks([4.0, 5.5]) == [4.0, 5.5]        # no process group
    # 2 replicas x 10 steps x 1 GB in 100 ms = 200 GB/s for the whole job
    assert bench.whole_job_gbs(2, 10, 1e9, 100.0) == pytest.approx(200.0)
    assert bench.whole_job_gbs(1, 10, 1e9, 100.0) == pytest.approx(100.0)


def test_reference_arm_prints_on_rank0_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        rc = bench.run_reference(types.SimpleNamespace(gpus=2, steps=1, warmup=0))
    assert rc == 0 and out.getvalue() == ""
