"""The replicated multi-GPU benchmark's only exchange -- slowest time and
summed work over ranks -- checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, iters = bench.reduce_over_ranks(100.0 + 50.0 * rank, 1000 + rank, device="cpu")
    q.put((rank, ms, iters))
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, iters in res:
        assert ms == 150.0 and iters == 2001.0


def test_single_process_is_identity():
    import bench
    assert bench.reduce_over_ranks(12.5, 7) == (12.5, 7.0)
