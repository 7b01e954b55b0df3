"""Host logic of bench.py's multi-process mode, on CPU with two gloo ranks: every rank reports the slowest rank's
time, the whole-job value counts the replica of every rank, and the reference arm runs on rank 0 only (the other
ranks return without work)."""
import argparse
import json
import os
import socket

import pytest

dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), LOCAL_RANK=str(rank),
                      WORLD_SIZE="2")
    import torch.distributed as d

    d.init_process_group("gloo", rank=rank, world_size=2)
    import bench

    ws, r, local = bench._dist()
    slowest = bench.max_over_ranks(10.0 + 5.0 * rank, ws, "cpu")  # rank 1 is the slow one
    value = bench.job_value(ws, 1000, slowest)
    d.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"ws": ws, "rank": r, "local": local, "slowest": slowest, "value": value}, f)
    d.destroy_process_group()


def test_two_ranks_slowest_time_and_job_value(tmp_path):
    import torch.multiprocessing as mp

    mp.spawn(_worker, args=(_free_port(), str(tmp_path)), nprocs=2, join=True)
    for rank in (0, 1):
        res = json.loads((tmp_path / f"rank{rank}.json").read_text())
        assert (res["ws"], res["rank"], res["local"]) == (2, rank, rank)
        assert res["slowest"] == 15.0
        assert res["value"] == pytest.approx(2 * 1000 / 15e-3)


def test_one_process_is_its_own_slowest():
    import bench

    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25
    assert bench.job_value(1, 4198401, 0.125) == pytest.approx(4198401 / 0.125e-3)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(argparse.Namespace(steps=1, warmup=3)) is None


def test_elastic_fp64_count_by_hand():
    """FP64 FMAs per point-step of the elastic step, counted by hand for 257 points per axis, 4 patches (M = 64),
    n_nb = 20: an x line sums junctions of 21, 41, 41, 41, 21 taps (165) for 6 derivatives; a y / z line's tiles
    sum (21 + 41) + (41 + 41) + (41 + 41) + (41 + 21) = 288 taps for 12 derivatives."""
    import bench

    assert abs(bench.elastic_dfma_per_point_step(256, 4, 20) - (6 * 165 + 12 * 288) / 257) < 1e-12
    # one patch per axis: only the two end junctions, one-sided
    assert abs(bench.elastic_dfma_per_point_step(64, 1, 8) - (6 * 18 + 12 * 34) / 65) < 1e-12
