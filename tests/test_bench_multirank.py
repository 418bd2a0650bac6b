"""Host logic of bench.py's multi-rank path on CPU with gloo (world size 2)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" 10 + r ms for 100 (r + 1) leaf-iterations
    ms, work = bench.aggregate(dist, 10.0 + rank, 100.0 * (rank + 1), torch.device("cpu"))
    out[rank] = (ms, work)
    dist.destroy_process_group()


def test_aggregate_max_time_sum_work():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # every rank sees the slowest rank's time and the total work
    assert res == {0: (11.0, 300.0), 1: (11.0, 300.0)}


def test_aggregate_single_process():
    import bench
    assert bench.aggregate(None, 12.5, 42, None) == (12.5, 42.0)
