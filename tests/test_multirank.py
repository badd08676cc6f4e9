"""The benchmark's multi-process path on CPU (gloo, world size 2): each rank
holds a replica and times its own batch; the job's time is the slowest rank's
and its throughput counts every rank's queries.  No GPU is needed: the same
helpers run over NCCL on GPUs."""
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


def _rank(rank, world, port, local_ms, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(local_ms[rank], dist, "cpu")
        out.put((rank, ms, bench.job_qps(world, 10_000, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_job_time():
    world, local_ms = 2, [39.5, 41.25]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, local_ms, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, qps in res:
        assert ms == pytest.approx(max(local_ms))
        assert qps == pytest.approx(world * 10_000 / max(local_ms) * 1e3)


def test_single_process_is_its_own_max():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_qps(1, 10_000, 40.0) == pytest.approx(250_000.0)
