"""The multi-rank path of bench.py on the CPU: two gloo ranks (127.0.0.1)
exercise the barrier and the max-over-ranks timing reduction that the GPU
bench uses for N > 1 replicas (no data-path collective exists: each rank
filters its own replica)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), FBF_BENCH_BACKEND="gloo")
    import bench

    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    bench.dist_barrier(w)
    total_ms = 10.0 + 5.0 * rank  # each rank's own timed total
    m = bench.dist_max(total_ms, w, None)
    bench.dist_barrier(w)
    q.put((rank, m))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 15.0), (1, 15.0)]


def test_single_rank_is_a_no_op():
    import bench

    assert bench.dist_max(3.5, 1) == 3.5
    bench.dist_barrier(1)
