"""The multi-rank path of bench.py on CPU: two gloo ranks decode disjoint frame shards (no data
exchange) and the job's throughput is the frames of all ranks over the slowest rank's time."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t_max, value = bench.aggregate(local_seconds=1.0 + rank, local_frames=100 * (rank + 1), info_bits=2048,
                                   dist=dist)
    out[rank] = (t_max, value)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_takes_slowest_rank_and_all_frames():
    world = 2
    port = _free_port()
    with tmp.Manager() as mgr:
        out = mgr.dict()
        tmp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t_max, value = res[r]
        assert t_max == pytest.approx(2.0)
        assert value == pytest.approx((100 + 200) * 2048 / 2.0 / 1e6)


def test_aggregate_single_process():
    import bench

    t, v = bench.aggregate(0.5, 1024, 2048)
    assert t == 0.5 and v == pytest.approx(1024 * 2048 / 0.5 / 1e6)
