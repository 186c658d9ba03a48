"""Parity at the full 192x192 brush size (n = 36865, G = 21.7 GB complex128) in the launch
configuration bench.py times (GreedyOptimizer, tensor-core update).  The oracle side is the
deferred FP64 oracle, which computes G entries one by one: every candidate's dFOM, the chosen
ids, all of E and the FOM are compared each step, and G on 4000 sampled entries plus the full
rows and columns of the flipped pixels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.lowrank import LowRankProblem
from paper_2202_05388_gb300 import build as BLD
from paper_2202_05388_gb300 import gfopt as B
from paper_2202_05388_gb300 import workloads as W
from paper_2202_05388_gb300.optimizer import GreedyOptimizer

from gpu_parity import GAP, TOL, compare_dfom, rel_err


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BLD.build()


def test_brush_192_full_size_three_steps():
    wl = W.brush_192()
    g = wl.geoms[0]
    lazy = LowRankProblem(g, wl.spec)
    opt = GreedyOptimizer(wl.geoms, wl.spec)
    opt.fill()
    rng = np.random.default_rng(2202)
    for t in range(3):
        opt.evaluate()
        d_orc = lazy.evaluate()
        compare_dfom(opt.dfom.cpu().numpy(), d_orc, tag=f"step {t}")
        ids = lazy.choose(d_orc)
        opt.select()
        r = opt.read_step()
        assert ids, "the 192x192 workload has improving brushes in its first steps"
        assert r.status == B.GF_OK
        if r.ids != ids:
            assert abs(d_orc[r.ids[0]] - d_orc[ids[0]]) <= GAP * abs(d_orc[ids[0]])
            opt.idx[0] = ids[0]
        opt.update()
        ids = lazy.accept(ids)
        torch.cuda.synchronize()
        assert abs(float(opt.fom.cpu()[0]) - lazy.fom()) <= TOL * lazy.fom()
        assert rel_err(opt.E[0].cpu().numpy(), lazy.E) <= TOL
        assert np.array_equal(opt.state.cpu().numpy(), lazy.state)
        i = rng.integers(0, g.n, 4000)
        j = rng.integers(0, g.n, 4000)
        Gs = opt.G[0][torch.as_tensor(i, device="cuda"), torch.as_tensor(j, device="cuda")].cpu().numpy()
        Gl = lazy.entries(i, j)
        scale = float(np.max(np.abs(lazy.rows(np.array([0])))))
        assert np.max(np.abs(Gs - Gl)) <= TOL * scale, f"step {t}: sampled G"
        V = np.flatnonzero(lazy.state != 0) if t == 0 else V_last
        Vt = torch.as_tensor(V, device="cuda")
        assert rel_err(opt.G[0][Vt, :g.n].cpu().numpy(), lazy.rows(V)) <= TOL
        assert rel_err(opt.G[0][:, Vt].cpu().numpy(), lazy.cols(V)) <= TOL
        V_last = np.array(sorted(set(np.flatnonzero(lazy.state != 0).tolist()) | set(V.tolist())))


# complex64 storage against the FP64 oracle: the lock-step bounds of the mixed-precision tests
C64_TOL = 2e-5
C64_DFOM = 1e-4


def _force(opt, ids, k):
    fixed = torch.full((k,), -1, dtype=torch.int32)
    fixed[:len(ids)] = torch.tensor(ids, dtype=torch.int32)
    opt.idx.copy_(fixed.to(opt.idx.device))
    opt.status.zero_()


def _sampled_G(opt, lazies, rng, tol, l_all=True):
    for l, lazy in enumerate(lazies):
        n = lazy.n
        i = rng.integers(0, n, 3000)
        j = rng.integers(0, n, 3000)
        Gs = opt.G[l][torch.as_tensor(i, device="cuda"), torch.as_tensor(j, device="cuda")].cpu().numpy()
        Gl = lazy.entries(i, j)
        scale = float(np.max(np.abs(lazy.rows(np.array([0])))))
        assert np.max(np.abs(Gs.astype(np.complex128) - Gl)) <= tol * scale


def test_brush_320_top32_c64_full_size_lockstep():
    """The 320x320 top-32 workload (n = 102401, complex64 G = 83.9 GB, rank-k p Woodbury on the
    tensor cores, streaming 128 x 256 tiles) for three steps from the oracle's choices: every candidate's
    dFOM, the applied set (joint decision), E, FOM and sampled G within the mixed-precision
    bounds of the FP64 oracle."""
    wl = W.brush_320_topk()
    g = wl.geoms[0]
    lazy = LowRankProblem(g, wl.spec)
    opt = GreedyOptimizer(wl.geoms, wl.spec, dtype="c64")
    opt.fill()
    rng = np.random.default_rng(3202)
    for t in range(3):
        opt.evaluate()
        d_orc = lazy.evaluate()
        d_gpu = opt.dfom.cpu().numpy()
        fin = np.isfinite(d_orc)
        assert np.array_equal(fin, np.isfinite(d_gpu))
        scale = max(1.0, float(np.max(np.abs(d_orc[fin]))))
        assert np.max(np.abs(d_gpu[fin] - d_orc[fin])) <= C64_DFOM * scale, t
        ids = lazy.choose(d_orc)
        assert ids
        _force(opt, ids, wl.spec.k)
        opt.update()
        lazy.accept(ids)
        torch.cuda.synchronize()
        assert int(opt.status.cpu()[0]) == B.GF_OK
        assert np.array_equal(opt.state.cpu().numpy(), lazy.state), t
        assert rel_err(opt.E[0].cpu().numpy(), lazy.E) <= C64_TOL, t
        assert abs(float(opt.fom.cpu()[0]) - lazy.fom()) <= C64_TOL * lazy.fom()
        _sampled_G(opt, [lazy], rng, C64_TOL)


def test_multilambda_c64_full_size_lockstep():
    """512x64 pixels at three wavelengths (complex64 G of 8.6 GB each, top-16 brushes): the
    summed dFOM of every candidate, the joint decision over all wavelengths, every wavelength's
    E and sampled G for three steps against one deferred FP64 oracle per wavelength."""
    wl = W.multi_lambda_512x64()
    lazies = [LowRankProblem(gg, wl.spec) for gg in wl.geoms]
    opt = GreedyOptimizer(wl.geoms, wl.spec, dtype="c64")
    opt.fill()
    rng = np.random.default_rng(512)
    from oracle import gf_oracle as O
    for t in range(3):
        opt.evaluate()
        d_orc = sum(lz.evaluate() for lz in lazies)
        d_gpu = opt.dfom.cpu().numpy()
        fin = np.isfinite(d_orc)
        assert np.array_equal(fin, np.isfinite(d_gpu))
        scale = max(1.0, float(np.max(np.abs(d_orc[fin]))))
        assert np.max(np.abs(d_gpu[fin] - d_orc[fin])) <= C64_DFOM * scale, t
        ids = O.select_topk(wl.geoms[0], wl.spec, d_orc)
        assert ids
        if len(ids) > 1 and not sum(lz.joint_dfom(ids) for lz in lazies) > 0.0:
            ids = ids[:1]
        _force(opt, ids, wl.spec.k)
        opt.update()
        for lz in lazies:
            lz.accept(ids, joint_check=False)
        torch.cuda.synchronize()
        assert int(opt.status.cpu()[0]) == B.GF_OK
        assert np.array_equal(opt.state.cpu().numpy(), lazies[0].state), t
        for l, lz in enumerate(lazies):
            assert rel_err(opt.E[l].cpu().numpy(), lz.E) <= C64_TOL, (t, l)
        fom = sum(lz.fom() for lz in lazies)
        assert abs(float(opt.fom.cpu()[0]) - fom) <= C64_TOL * fom
        _sampled_G(opt, lazies, rng, C64_TOL)


def test_batch_48_full_size_sampled_problems():
    """The 48 seeded problems (sum of G = 76.6 GB complex128) advanced by the fused batch
    schedule for three steps; four of them (the two largest and two others) are replayed by
    the deferred FP64 oracle: choices, E, FOM and sampled G within 1e-10."""
    from paper_2202_05388_gb300.batch import BatchOptimizer
    wls = W.batch_48()
    bo = BatchOptimizer(wls)
    assert bo.schedule.fused
    bo.fill()
    bo.capture(2)                                   # + one step before the capture
    bo.replay()
    torch.cuda.synchronize()
    order = sorted(range(len(wls)), key=lambda i: -bo.sizes[i])
    picks = order[:2] + [order[len(order) // 2], order[-1]]
    rng = np.random.default_rng(48)
    for i in picks:
        wl = wls[i]
        lazy = LowRankProblem(wl.geoms[0], wl.spec)
        for _ in range(3):
            d = lazy.evaluate()
            ids = lazy.choose(d)
            if not ids:
                break
            lazy.accept(ids)
        opt = bo.opts[i]
        assert np.array_equal(opt.state.cpu().numpy(), lazy.state), i
        assert rel_err(opt.E[0].cpu().numpy(), lazy.E) <= TOL, i
        assert abs(float(opt.fom.cpu()[0]) - lazy.fom()) <= TOL * lazy.fom()
        _sampled_G(opt, [lazy], rng, TOL)


def test_resident_a_update_groups_and_segments_lockstep():
    """215x215 brushes, top-8 (joint rank <= 32: every update in the resident-A form), complex64
    G = 17 GB, three lock-step steps against the deferred FP64 oracle.  n = 46226 gives 362 row
    tiles: two full groups of 152 (each CTA one row tile across all 723 column tiles, the CTAs in
    step) and a last group of 58 row tiles cut into two column segments each -- every tile
    schedule of the kernel at a size the oracle still samples quickly."""
    g = W.small(215, 215, kind=W.KIND_BRUSH2, dir_mask=3, k=8, excl_radius=3, dtype="c64").geoms[0]
    spec = W.CandidateSpec(W.KIND_BRUSH2, 3, 8, 3)
    assert g.N + 1 == 46226
    lazy = LowRankProblem(g, spec)
    opt = GreedyOptimizer((g,), spec, dtype="c64")
    opt.fill()
    rng = np.random.default_rng(4215)
    for t in range(3):
        opt.evaluate()
        d_orc = lazy.evaluate()
        d_gpu = opt.dfom.cpu().numpy()
        fin = np.isfinite(d_orc)
        assert np.array_equal(fin, np.isfinite(d_gpu))
        scale = max(1.0, float(np.max(np.abs(d_orc[fin]))))
        assert np.max(np.abs(d_gpu[fin] - d_orc[fin])) <= C64_DFOM * scale, t
        ids = lazy.choose(d_orc)
        assert ids
        _force(opt, ids, spec.k)
        opt.update()
        lazy.accept(ids)
        torch.cuda.synchronize()
        assert int(opt.status.cpu()[0]) == B.GF_OK
        assert np.array_equal(opt.state.cpu().numpy(), lazy.state), t
        assert rel_err(opt.E[0].cpu().numpy(), lazy.E) <= C64_TOL, t
        assert abs(float(opt.fom.cpu()[0]) - lazy.fom()) <= C64_TOL * lazy.fom()
        _sampled_G(opt, [lazy], rng, C64_TOL)
        # whole rows in each part of the schedule: full groups, and the segmented last group
        rows = np.array([5, 128 * 151 + 3, 128 * 200 + 77, 128 * 310 + 1, g.N])
        Gr = opt.G[0][torch.as_tensor(rows, device="cuda"), :g.N + 1].cpu().numpy().astype(np.complex128)
        Gl = lazy.rows(rows)
        assert np.max(np.abs(Gr - Gl)) <= C64_TOL * float(np.max(np.abs(Gl))), t
