"""The benchmark's multi-process plumbing (replicas: one process per GPU, a
barrier and the max over ranks of the timed region, no data-path collective)
on two CPU processes over gloo."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank: int, world: int, port: int, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, local, w = bench.dist_init("gloo")
    bench.barrier(w)
    slowest = bench.max_over_ranks(1.0 + rank, w)        # the job's time is its slowest rank's
    frames = w * 10                                          # weak scaling: units of all ranks
    # the reference arm runs on rank 0 only; the other ranks leave at once
    skipped = rank != 0 and bench.run_reference(None) == 0
    out.put((r, local, w, slowest, frames / slowest, skipped))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_over_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    assert all(r[2] == world for r in res)
    assert all(r[3] == 2.0 for r in res)          # max over ranks, seen by every rank
    assert all(r[4] == 10.0 for r in res)         # 20 frames in the slowest rank's 2.0 s
    assert res[1][5] and not res[0][5]


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)
