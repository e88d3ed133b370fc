"""The multi-GPU path is replicas only (one image or batch per rank, no
collective on the data path): the bench's whole-job aggregation over ranks,
checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r processed (r + 1) * 1e6 units in (10 + 5 r) ms
    value, ms = bench.aggregate((rank + 1) * 1e6, 10.0 + 5.0 * rank, world)
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # units summed over ranks (3e6), divided by the slowest rank's 15 ms
    for r in range(world):
        value, ms = res[r]
        assert ms == pytest.approx(15.0)
        assert value == pytest.approx(3e6 / 15e-3 / 1e6)


def test_aggregate_single_rank():
    import bench
    value, ms = bench.aggregate(2e6, 4.0, 1)
    assert ms == 4.0 and value == pytest.approx(2e6 / 4e-3 / 1e6)
