"""The multi-GPU bench's host logic on two CPU ranks (gloo, no GPU).

bench.py with N GPUs runs one independent realisation per rank (seed +
rank), brackets the timed region with barriers, takes the slowest rank's
time and reports all ranks' work over it ("weak" scaling).  These tests run
exactly those helpers on two gloo ranks, and check that the reference arm
does its work on rank 0 only.
"""

import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import bench
    from paper_2005_02498_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        net = W.large_loop_network(seed=bench.rank_seed(rank))
        dist.barrier()
        elapsed = 1.0 + 0.5 * rank  # the ranks finish at different times
        slowest = bench.max_over_ranks(elapsed, dist, "cpu")
        value = bench.whole_job_rate(net.n_nodes ** 2 * 10, world, slowest)
        np.save(os.path.join(out_dir, "rank%d.npy" % rank),
                np.array([slowest, value, net.xyz[0, 0], net.n_nodes]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_weak_scaling_helpers(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [np.load(tmp_path / ("rank%d.npy" % k)) for k in range(world)]
    # every rank sees the slowest rank's time and the same whole-job value
    assert r[0][0] == r[1][0] == 1.5
    assert r[0][1] == r[1][1] == pytest.approx(2 * 32768 ** 2 * 10 / 1.5)
    # the ranks ran different realisations of the same size
    assert r[0][3] == r[1][3] == 32768
    assert r[0][2] != r[1][2]


def test_single_process_helpers_need_no_process_group():
    import bench
    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
    assert bench.rank_seed(0) != bench.rank_seed(1)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                                      "--warmup", "0"])
    assert bench.main() == 0
    assert capsys.readouterr().out == ""  # rank 1 prints nothing and does no work
