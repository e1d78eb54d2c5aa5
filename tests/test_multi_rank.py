"""Host logic of the multi-GPU benchmark path (one replica per rank, no
collective on the data path; the slowest rank's time) with world_size-2 gloo
process groups on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(world, 10.0 + 5.0 * rank)   # rank 1 is slower
    bench.barrier(world)
    q.put((rank, ms, bench.weak_value(world, 1000, ms)))
    dist.destroy_process_group()


def test_two_ranks_take_slowest_time_and_sum_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]            # both see the max
    assert out[0][2] == pytest.approx(2 * 1000 / 0.015)    # all ranks' units / slowest time


def _ref_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import contextlib
    import io
    import bench
    buf = io.StringIO()

    class A:
        workload = "planar_8x7"
        steps = 1
        warmup = 0
        gpus = world
    with contextlib.redirect_stdout(buf):
        if rank != 0:
            bench.run_reference(A, world, rank)
    q.put((rank, buf.getvalue()))


def test_reference_arm_other_ranks_exit_without_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    p = ctx.Process(target=_ref_worker, args=(1, 2, port, q))
    p.start()
    rank, text = q.get(timeout=120)
    p.join(timeout=60)
    assert p.exitcode == 0 and rank == 1 and text == ""
