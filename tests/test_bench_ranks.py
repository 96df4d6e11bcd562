"""The benchmark's multi-rank aggregation (one replica per GPU: the slowest
rank's time, the whole job's pairs), run as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took (r + 1) ms and 2.5 (r + 1) ms end to end and counted 1000 (r + 1) pairs
    mx, sm = bench.reduce_over_ranks([1.0 * (rank + 1), 2.5 * (rank + 1)],
                                     [1000.0 * (rank + 1), 10.0], "cpu")
    out[rank] = (mx, sm)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_slowest_time_and_total_pairs():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        mx, sm = res[r]
        assert mx == [2.0, 5.0]
        assert sm == [3000.0, 20.0]
