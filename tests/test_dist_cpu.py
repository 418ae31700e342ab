"""Multi-process path of bench.py on CPU: two gloo ranks (127.0.0.1) agree on the slowest
rank's time and on the whole-job value (replicas: every rank advances its own mesh)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    secs = [1.5, 2.5][rank]
    m = bench.reduce_max(secs, world, device="cpu")
    q.put((rank, m, bench.job_value(world, 1000, 10, m)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_and_value():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.5, 2.5]
    assert res[0][2] == pytest.approx(2 * 1000 * 10 / 2.5)


def test_single_rank_is_identity():
    import bench

    assert bench.reduce_max(3.0, 1) == 3.0
    assert bench.job_value(1, 4096, 5, 2.0) == 4096 * 5 / 2.0
