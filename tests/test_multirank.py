"""The multi-GPU path on CPU: replicas only.

Every rank solves its own copy of the workload and no collective touches the
data path; the only cross-rank step is the benchmark's aggregation (the job
takes as long as the slowest rank, and moves the bytes of all ranks).  Two
gloo ranks on the host check that step, with unequal per-rank figures.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = [120.0, 150.0][rank]
        local_bytes = [3.0e9, 5.0e9][rank]
        out[rank] = bench.job_throughput(local_ms, local_bytes, dist, None)
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        ms, byt, gbs = out[r]
        assert ms == 150.0  # the slowest rank
        assert byt == 8.0e9  # both ranks' bytes
        assert gbs == pytest.approx(8.0e9 / 0.150 / 1e9)


def test_single_process_needs_no_group():
    import bench
    ms, byt, gbs = bench.job_throughput(200.0, 4.0e9)
    assert (ms, byt) == (200.0, 4.0e9) and gbs == pytest.approx(20.0)
