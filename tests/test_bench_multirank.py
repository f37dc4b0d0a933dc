"""The multi-rank leg of bench.py on CPU: two gloo ranks, each with its own
replica; the job time is the slowest rank's and the throughput counts the
cells of all ranks (weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, glups = bench.aggregate(100.0 + 50.0 * rank, cells_per_rank=1000, steps=10, world=world, device="cpu")
    q.put((rank, ms, glups))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(60)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(2))
    for _, ms, glups in out:
        assert ms == 150.0
        assert abs(glups - 2 * 1000 * 10 / 0.150 / 1e9) < 1e-15
