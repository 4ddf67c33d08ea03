"""The N > 1 path of bench.py is replicas: every rank sketches its own matrix
and only the timing is combined (the slowest rank's time, every rank's
sketches). The combination runs here on two gloo ranks on the CPU."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        total_ms = bench.rank_max(10.0 + 5.0 * rank)  # rank 1 is the slow one
        steps = int(bench.rank_max(7 + rank))         # ranks agree on the step count
        value = bench.job_value(world, 4, 10, total_ms)
        dist.barrier()
        q.put((rank, total_ms, steps, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_timing():
    pytest.importorskip("torch")
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
    for rank, total_ms, steps, value in out:
        assert total_ms == 15.0 and steps == 8
        assert value == pytest.approx(2 * 4 * 10 / 0.015)


def test_single_process_is_identity():
    import bench
    assert bench.rank_max(3.5) == 3.5
    assert bench.job_value(1, 4, 5, 1000.0) == pytest.approx(20.0)
