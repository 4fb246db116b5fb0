"""The benchmark's multi-GPU form is replicas only: every rank advances its own
plasma and the ranks meet only in a barrier and a max of the elapsed time.
That host logic runs here on two CPU ranks over gloo."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms = bench.reduce_max(10.0 + 5.0 * rank, dist, "cpu")      # rank 1 is the slow one
    value = bench.replica_value(1000, world, 4, ms)
    out.put((rank, ms, value))
    dist.destroy_process_group()


def test_replicas_reduce_to_slowest_rank_over_gloo():
    import torch.multiprocessing as mp
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
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == pytest.approx(1000 * 2 * 4 / 15e-3)


def test_single_rank_without_process_group():
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
    assert bench.replica_value(10, 1, 2, 1.0) == pytest.approx(2e4)
