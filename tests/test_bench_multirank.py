"""bench.py's multi-rank aggregation (N independent replicas, weak scaling) with two
gloo ranks on the CPU: units add up, the time is the slowest rank's."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist            # noqa: E402
import torch.multiprocessing as mp          # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units, ms = bench.aggregate(1000.0 * (rank + 1), 10.0 + 5.0 * rank, dist, "cpu")
    q.put((rank, units, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for _, units, ms in out:
        assert units == 3000.0 and ms == 15.0
    # whole-job throughput = all units over the slowest rank
    assert 3000.0 / (15.0 / 1000.0) == 200000.0


def test_single_process_aggregate_is_identity():
    import bench
    assert bench.aggregate(5.0, 2.0) == (5.0, 2.0)
