"""Host-side logic of multi-GPU runs on CPU with two gloo ranks: the batch is
dealt without overlap or gaps, and the end-of-run combination takes the
slowest rank's time and the sum of the work."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2001_11533_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = replicas.deal(16, rank, world)
        t = 1.0 + rank            # rank 1 is the slow one
        work = 10 * (rank + 1)
        mx, sm = replicas.combine([t, 0.5 * rank], [work, len(mine)])
        out[rank] = (mine, mx, sm)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    shares = [set(res[r][0]) for r in range(world)]
    assert shares[0].isdisjoint(shares[1]) and shares[0] | shares[1] == set(range(16))
    for r in range(world):
        _, mx, sm = res[r]
        assert mx == [2.0, 0.5]               # the slowest rank's time
        assert sm == [30.0, 16.0]             # all work, all problems


def test_single_process_and_arguments():
    assert replicas.deal(5, 0, 1) == [0, 1, 2, 3, 4]
    assert replicas.deal(5, 1, 2) == [1, 3]
    assert replicas.combine([1.5], [3]) == ([1.5], [3.0])
    with pytest.raises(ValueError):
        replicas.deal(4, 2, 2)
