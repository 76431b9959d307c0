"""The multi-GPU path of bench.py on CPU: two gloo ranks.

The method runs one lattice per GPU with no exchange between them (replicas),
so the only multi-rank logic is the max-over-ranks time and the whole-job
value; both are checked here with world_size 2 over gloo.
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
    slowest = bench.reduce_max(10.0 + 5.0 * rank, torch.device("cpu"))
    value = bench.replica_value(2048 * 2048, 100, world, slowest / 1e3)
    dist.barrier()
    out[rank] = (slowest, value)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        slowest, value = res[r]
        assert slowest == 15.0
        assert value == pytest.approx(2048 * 2048 * 100 * 2 / 0.015 / 1e6)

