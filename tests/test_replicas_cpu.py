"""Multi-GPU host logic of bench.py on CPU: replicas with no data-path
collective, max-over-ranks timing, whole-job frames/s (gloo, world size 2)."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [10.0 + 5.0 * rank, 3.0 - rank, 7.0]
    got = bench.reduce_max_over_ranks(local, dist)
    value = bench.replicas_value(128 * 10, world, got[0])
    out.put((rank, got, value))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value in res:
        assert got == [15.0, 3.0, 7.0]           # element-wise max over the two ranks
        assert value == pytest.approx(128 * 10 * 2 / 0.015)  # all frames over the slowest rank's time


def test_single_process_reduction_is_identity():
    assert bench.reduce_max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    assert bench.replicas_value(100, 1, 1000.0) == pytest.approx(100.0)


def test_reference_arm_nonzero_ranks_do_no_work():
    class A:
        steps, warmup, gpus = 1, 3, 2
    assert bench.run_reference(A(), rank=1, world=2) == 0
