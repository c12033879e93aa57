"""Replica runs (one independent problem per rank, no collective on the data
path): the bench's timing aggregation over two gloo ranks on the CPU (every
rank learns the slowest replica's time after the barrier), the reference
arm's rank handling (rank 0 alone works and prints; the others exit 0), and
the keys of the reference arm's JSON line."""
import argparse
import socket

import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench.rank_barrier(dist, cuda=False)
        out[rank] = bench.max_over_ranks(1.5 + 2.0 * rank, dist, device="cpu")
        bench.rank_barrier(dist, cuda=False)
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
        assert dict(out) == {0: 3.5, 1: 3.5}


def test_single_process_aggregation_is_the_value():
    assert bench.max_over_ranks(0.25, None) == 0.25


def test_reference_arm_runs_on_rank_zero_only(capsys):
    args = argparse.Namespace(steps=1, warmup=0, gpus=2, ref_iters=86)
    assert bench.run_reference(args, 1, 2) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_json_line(capsys):
    """The reference arm's one JSON line (the oracle timed on the host cores) has
    the keys the benchmark contract names, the main arm's metric and unit, and
    an e2e object with no host-device traffic."""
    import json
    args = argparse.Namespace(steps=1, warmup=0, gpus=1, ref_iters=86)
    assert bench.run_reference(args, 0, 1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "s"
    assert line["higher_is_better"] is False and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
