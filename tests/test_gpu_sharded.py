"""Row-block shards of G on the GPU (gf_shard_* calls, paper Sec. III's partitioned form) against the
FP64 oracle.  Two or three shards of one problem live on cuda:0; the collectives between them (max
of the dFOM arrays, sum of the row panels, the halo exchange) are done here in the test process,
and the shards follow the oracle's choices lock-step: every step compares the merged dFOM array,
then each shard's rows of G, E, the state and the FOM.  The last test runs the real driver
(ShardedOptimizer) in two processes on cuda:0 over gloo."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import gf_oracle as O
from paper_2202_05388_gb300 import build as BLD
from paper_2202_05388_gb300 import gfopt as B
from paper_2202_05388_gb300 import workloads as W
from paper_2202_05388_gb300.sharded import split_rows

from gpu_parity import TOL, rel_err

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BLD.build()


def _shards(wl, dtype, world, algo=None):
    from paper_2202_05388_gb300.sharded import LibShard
    g = wl.geoms[0]
    h = B.Handle(0)
    if algo is not None:
        h.gf_set_update_algo(algo)
    out = [LibShard(g, wl.spec, dtype, y0, y1, handle=h) for y0, y1 in split_rows(g.ny, world)]
    for s in out:
        s.fill()
    _halo(out)
    return out


def _halo(shards):
    recs = [s.pack_halo().clone() for s in shards]
    for r, s in enumerate(shards[:-1]):
        s.unpack_halo(recs[r + 1])


def _apply_ids(shards, ids, spec=None):
    k = (spec or shards[0].spec).k
    for s in shards:
        s.idx.fill_(-1)
        s.idx[:len(ids)] = torch.tensor(ids, dtype=torch.int32, device=s.idx.device)
        s.status.zero_()
        s.gather(spec)
    total = torch.zeros_like(shards[0].panel)
    for s in shards:
        total += s.panel
    for s in shards:
        s.panel.copy_(total)
        s.apply(spec)
    _halo(shards)
    assert k >= len(ids)


def _reach(shards, orc, state):
    """Forced single-pixel flips on the shards and on the oracle (one at a time)."""
    single = W.CandidateSpec(W.KIND_SINGLE, W.DIR_FILL | W.DIR_CLEAR, 1)
    for j in np.flatnonzero(state):
        _apply_ids(shards, [int(j)], single)
        V, d = O.candidate(orc.geoms[0], single, orc.state, int(j))
        Gn, En, ok = O.apply_update(orc.Gs[0], orc.Es[0], V, d)
        assert ok
        orc.Gs, orc.Es = [Gn], [En]
        orc.state[V] ^= 1


def _compare(shards, orc, tol, tag):
    torch.cuda.synchronize()
    for s in shards:
        G = s.G[:, :s.n].cpu().numpy().astype(np.complex128)
        r0 = s.y0 * s.geom.nx
        assert rel_err(G, orc.Gs[0][r0:r0 + s.rows]) <= tol, f"{tag} shard {s.y0}-{s.y1} G"
        assert rel_err(s.E.cpu().numpy(), orc.Es[0]) <= tol, f"{tag} E"
        assert np.array_equal(s.state.cpu().numpy(), orc.state), f"{tag} state"
        assert abs(float(s.fom.cpu()[0]) - orc.fom()) <= tol * orc.fom(), f"{tag} FOM"


@pytest.mark.parametrize("nx,ny,kind,k,dtype,world,algo,seed,steps", [
    (12, 11, W.KIND_BRUSH2, 1, "c128", 2, B.GF_UPDATE_TENSOR, 31, 4),    # tensor-core digit update, p <= 4
    (12, 11, W.KIND_BRUSH2, 1, "c128", 3, None, 32, 4),                  # FP64 FMA at this size
    (14, 12, W.KIND_BRUSH2, 4, "c128", 2, None, 33, 3),                  # top-4: joint rank up to 16
    (10, 9, W.KIND_SINGLE, 1, "c128", 2, B.GF_UPDATE_TENSOR, 34, 4),
    (14, 12, W.KIND_BRUSH2, 1, "c64", 2, None, 35, 4),                   # FP32 stream, p <= 4
    (20, 18, W.KIND_BRUSH2, 4, "c64", 2, None, 36, 3),                   # split-FP16 tensor cores
])
def test_shards_lockstep_with_the_oracle(nx, ny, kind, k, dtype, world, algo, seed, steps):
    wl = W.small(nx, ny, kind=kind, dir_mask=3, k=k, excl_radius=3, dtype=dtype)
    g = wl.geoms[0]
    orc = O.OracleProblem(wl.geoms, wl.spec)
    shards = _shards(wl, dtype, world, algo)
    tol = TOL if dtype == "c128" else 2e-5
    _compare(shards, orc, tol, "fill")
    _reach(shards, orc, W.random_state(g.N, seed=seed, fill=0.3))
    _compare(shards, orc, tol, "patterned start")
    for t in range(steps):
        for s in shards:
            s.evaluate()
        merged = shards[0].dfom.clone()
        for s in shards[1:]:
            merged = torch.maximum(merged, s.dfom)
        d_gpu = merged.cpu().numpy()
        d_orc = orc.evaluate()
        fin = np.isfinite(d_orc)
        assert np.array_equal(fin, np.isfinite(d_gpu)), t
        scale = max(1.0, float(np.max(np.abs(d_orc[fin]))))
        assert np.max(np.abs(d_gpu[fin] - d_orc[fin])) <= (TOL if dtype == "c128" else 1e-4) * scale, t
        ids = orc.choose(d_orc)
        if not ids:
            break
        _apply_ids(shards, ids)
        orc.accept(ids)
        _compare(shards, orc, tol, f"step {t}")


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, steps, out):
    import torch.distributed as dist
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from paper_2202_05388_gb300 import workloads as W2
    from paper_2202_05388_gb300.sharded import ShardedOptimizer
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        wl = W2.small(16, 14, kind=W2.KIND_BRUSH2, dir_mask=3, k=3, excl_radius=2)
        opt = ShardedOptimizer(wl.geoms[0], wl.spec, dtype="c128")
        opt.fill()
        res = opt.run(steps)
        torch.cuda.synchronize()
        G = opt.shard.G[:, :opt.shard.n].cpu().numpy()
        out[rank] = ([(r.ids, r.fom, r.status) for r in res], G, opt.shard.y0, opt.shard.rows)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_sharded_driver_two_processes_on_one_gpu():
    import torch.multiprocessing as mp
    world, steps = 2, 5
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, _free_port(), steps, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    wl = W.small(16, 14, kind=W.KIND_BRUSH2, dir_mask=3, k=3, excl_radius=2)
    orc = O.OracleProblem(wl.geoms, wl.spec)
    ref = []
    for _ in range(steps):
        ids = orc.choose(orc.evaluate())
        if not ids:
            break
        orc.accept(ids)
        ref.append((ids, orc.fom()))
    for r in range(world):
        traj, G, y0, rows = res[r]
        assert [t[0] for t in traj[:len(ref)]] == [x[0] for x in ref]
        for (ids, fom, st), (ids_o, fom_o) in zip(traj, ref):
            assert st == B.GF_OK and abs(fom - fom_o) <= TOL * fom_o
        r0 = y0 * wl.geoms[0].nx
        assert rel_err(G, orc.Gs[0][r0:r0 + rows]) <= TOL
