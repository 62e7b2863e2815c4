"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1) reduce
their timed region to the slowest rank's time and sum their work; each rank
gets its own ensemble seed (weak scaling, no data-path collective)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t, v = bench.aggregate(1.0 + rank, 100.0 * (rank + 1), ws, dist)
    out[rank] = (t, v, bench.rank_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    # slowest rank: 2.0 s; total work 100 + 200
    for rank in range(ws):
        t, v, seed = res[rank]
        assert t == 2.0 and v == pytest.approx(300.0 / 2.0)
    assert res[0][2] != res[1][2]


def test_single_rank_aggregation():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(2.0, 50.0, 1) == (2.0, 25.0)
