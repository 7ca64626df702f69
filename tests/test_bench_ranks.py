"""The bench's multi-rank path on CPU: two gloo ranks (world size 2), each
timing its own replica; the reported step time is the slowest rank's and the
job throughput counts both replicas (weak scaling)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench._dist()
        local_ms = 10.0 + 5.0 * rank          # rank 1 is the slower one
        ms = bench._max_over_ranks(local_ms)
        q.put((r, ws, local, ms, bench._job_gteps(ws, 1000, 50, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, (r, ws, local, ms, gteps) in enumerate(res):
        assert (r, ws, local) == (rank, 2, rank)
        assert ms == 15.0                                    # the slowest rank's time on every rank
        assert gteps == pytest.approx(2 * 1000 * 50 / 15e-3 / 1e9)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench._max_over_ranks(3.5) == 3.5
    assert bench._job_gteps(1, 10, 5, 2.0) == pytest.approx(10 * 5 / 2e-3 / 1e9)
