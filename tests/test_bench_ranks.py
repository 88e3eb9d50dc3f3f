"""bench.py's multi-rank aggregation, run as two gloo ranks on the CPU.

Replicas: each rank solves its own LPs; whole-job throughput is all ranks'
pivots over the slowest rank's time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mx, sm = bench.reduce_over_ranks(dist, [10.0 + rank, -rank], [100.0 * (rank + 1), 1.0])
    out.put((rank, mx, sm))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, mx, sm in res:
        assert mx == [11.0, 0.0]
        assert sm == [300.0, 2.0]


def test_reduce_over_ranks_single_process_identity():
    import bench
    assert bench.reduce_over_ranks(None, [3.0], [4.0]) == ([3.0], [4.0])
