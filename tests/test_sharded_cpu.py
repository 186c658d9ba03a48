"""The row-sharded driver (paper_2202_05388_gb300/sharded.py) on two gloo ranks on the CPU: each rank
holds one band of G's rows in an oracle-backed shard (tests/shard_fake.py), and the driver's
collectives -- the max of the dFOM arrays, the sum of the row panels, the halo all-gather -- must
reproduce the unsharded oracle's trajectory (same choices, FOM within 1e-12)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import gf_oracle as O
from paper_2202_05388_gb300 import workloads as W
from paper_2202_05388_gb300.sharded import split_rows

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_split_rows_covers_every_pixel_row_once():
    for ny in (2, 7, 64, 320):
        for world in range(1, min(ny, 9) + 1):
            bands = split_rows(ny, world)
            assert len(bands) == world and bands[0][0] == 0 and bands[-1][1] == ny
            assert all(a[1] == b[0] for a, b in zip(bands, bands[1:]))
            h = [y1 - y0 for y0, y1 in bands]
            assert min(h) >= 1 and max(h) - min(h) <= 1
    with pytest.raises(ValueError):
        split_rows(3, 4)


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, case, steps, out):
    import torch.distributed as dist
    for p in (ROOT, os.path.join(ROOT, "tests")):
        if p not in sys.path:
            sys.path.insert(0, p)
    from paper_2202_05388_gb300.sharded import Comm, ShardedOptimizer, split_rows
    from shard_fake import OracleShard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        wl = _workload(case)
        g = wl.geoms[0]
        y0, y1 = split_rows(g.ny, world)[rank]
        comm = Comm()
        opt = ShardedOptimizer(g, wl.spec, comm=comm, shard=OracleShard(g, wl.spec, y0, y1))
        opt.fill()
        res = opt.run(steps)
        out[rank] = [(r.ids, r.fom, r.status) for r in res]
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _workload(case):
    if case == "brush_k1":
        return W.small(9, 8, kind=W.KIND_BRUSH2, dir_mask=3)
    if case == "brush_top3":
        return W.small(11, 10, kind=W.KIND_BRUSH2, dir_mask=3, k=3, excl_radius=2)
    return W.small(8, 7, kind=W.KIND_SINGLE, dir_mask=3)


@pytest.mark.parametrize("case,world,steps", [("brush_k1", 2, 6), ("brush_top3", 2, 4), ("single", 3, 6)])
def test_sharded_driver_matches_the_unsharded_oracle(case, world, steps):
    import torch.multiprocessing as mp
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), case, steps, out), nprocs=world, join=True)
        res = dict(out)
    wl = _workload(case)
    orc = O.OracleProblem(wl.geoms, wl.spec)
    ref = []
    for _ in range(steps):
        ids = orc.choose(orc.evaluate())
        if not ids:
            ref.append(([], orc.fom(), 4))
            break
        orc.accept(ids)
        ref.append((ids, orc.fom(), 0))
    for r in range(world):
        got = res[r]
        assert len(got) == len(ref)
        for (ids_g, fom_g, st_g), (ids_o, fom_o, st_o) in zip(got, ref):
            assert st_g == st_o
            assert ids_g == ids_o
            assert abs(fom_g - fom_o) <= 1e-12 * max(1.0, fom_o)
