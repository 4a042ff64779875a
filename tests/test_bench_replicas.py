"""The multi-GPU bookkeeping of bench.py (one replica per rank, barrier,
max-over-ranks time, whole-job throughput) on two CPU processes over gloo,
and the reference arm's behaviour on ranks other than 0."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    rep = bench.Replicas("gloo", "cpu")
    rep.barrier()
    t = 1.0 + rank                        # rank r "took" 1 + r seconds
    out[rank] = (rep.maxed(t), rep.throughput(1000.0, rep.maxed(t)), rep.world)
    rep.barrier()
    rep.close()


def test_two_ranks_max_time_and_whole_job_throughput():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        tmax, thr, w = out[r]
        assert w == world
        assert tmax == 2.0                # every rank sees the slowest rank's time
        assert thr == pytest.approx(world * 1000.0 / 2.0)


def test_single_process_is_its_own_job():
    for k in ("RANK", "WORLD_SIZE"):
        os.environ.pop(k, None)
    sys.path.insert(0, ROOT)
    import bench
    rep = bench.Replicas("gloo", "cpu")
    assert rep.world == 1 and rep.maxed(3.5) == 3.5 and rep.throughput(10.0, 2.0) == 5.0


def test_reference_arm_does_no_work_on_other_ranks(capsys):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(steps=3, warmup=3, grid=1024)
    assert bench.run_reference(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""
