"""The benchmark's multi-rank path on CPU: two gloo ranks on 127.0.0.1 run
independent replicas; the job time is the slowest rank's and the throughput
counts every rank's units (replicas only, no collective on the data path)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 1.0 + rank * 0.5  # rank 1 is slower
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    value = bench.job_throughput(world, 524288, ms)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms, value))


def test_two_rank_replicas_gloo():
    mp = pytest.importorskip("torch.multiprocessing")
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
    for rank, ms, value in res:
        assert ms == 1.5  # the slowest rank sets the job time on every rank
        assert abs(value - 2 * 524288 / 1.5e-3 / 1e6) < 1e-9
