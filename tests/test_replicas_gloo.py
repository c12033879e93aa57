"""Replica runs (one independent problem per rank, no collective on the data
path): the bench's timing aggregation over two gloo ranks on the CPU (every
rank learns the slowest replica's time after the barrier), and the reference
arm's rank handling (rank 0 alone works and prints; the others exit 0)."""
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
