"""The multi-GPU path of bench.py, on CPU with two gloo ranks.

Under torchrun every rank solves a batch of its own: no collective touches the
data path, and the timing takes the slowest rank. These tests check that host
logic without a GPU: the ranks' batches are disjoint, the reduction gives
every rank the maximum time, the whole-job throughput counts all ranks' solves
over that time, and the reference arm runs on rank 0 only.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    import workloads as w
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        count = 16
        shapes = w.banded_batch_shapes(count, bench.rank_seed0(rank, count))
        seeds = sorted(s for _, _, s in shapes)
        all_seeds = [None] * world
        dist.all_gather_object(all_seeds, seeds)
        ms_local = 100.0 + 50.0 * rank  # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms_local, dist, "cpu")
        value = bench.job_throughput(count, world, 3, ms_max)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(repr({"seeds": all_seeds, "ms_max": ms_max, "value": value}))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    res = [eval(open(tmp_path / f"rank{r}.txt").read()) for r in range(world)]
    for r in res:
        assert r["ms_max"] == 150.0               # the slowest rank's time, on every rank
        assert r["value"] == 16 * 2 * 3 / 0.150   # all ranks' solves over that time
    s0, s1 = res[0]["seeds"]
    assert s0 and s1 and not set(s0) & set(s1)   # disjoint batches
    assert res[0]["seeds"] == res[1]["seeds"]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(ref_sample=8, warmup=3, steps=5, gpus=2)
    assert bench.run_reference(args) == 0  # returns at once, no oracle work


def test_single_process_reduction_is_the_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(512, 1, 5, 1000.0) == 2560.0


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """Rank 0 times the oracle on a bounded sample and prints one JSON line
    with the keys the benchmark contract asks of the reference arm."""
    import argparse
    import json
    import bench
    monkeypatch.setenv("RANK", "0")
    args = argparse.Namespace(ref_sample=2, warmup=0, steps=1, gpus=1)
    assert bench.run_reference(args) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] == d["e2e"]["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == bench.WORKLOAD
