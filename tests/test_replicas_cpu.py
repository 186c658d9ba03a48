"""The multi-GPU mode of bench.py is independent replicas, one per rank (the path has no exchange
step): the reported throughput is the flips of all ranks over the slowest rank's time.  Checked
here with two gloo ranks on the CPU: the rank environment and the aggregation bench.py runs."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    assert bench.dist_env() == (rank, world, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r ran 3 (r + 1) flips in 10 + 5 r ms
        out[rank] = bench.reduce_replicas(10.0 + 5.0 * rank, 3 * (rank + 1), "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_aggregate_over_gloo():
    import torch.multiprocessing as mp
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (15.0, 9)      # slowest rank's time, flips of both ranks
