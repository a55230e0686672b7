"""The N > 1 path of bench.py (replicas: one process per GPU, no data-path collective) on
two CPU processes over gloo: rendezvous on 127.0.0.1, the barrier, and the max over
ranks that the job's timing takes."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), PFMP_BENCH_GLOO="1")
    import torch.distributed as dist

    import bench

    r, w = bench.dist_setup(world)
    v = bench.allmax(10.0 + 5.0 * r, w)
    bench.barrier(w)
    q.put((r, w, v))
    dist.destroy_process_group()


def test_two_ranks_barrier_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 15.0), (1, 2, 15.0)]
