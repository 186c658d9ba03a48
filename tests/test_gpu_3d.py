"""The 3-D (dyadic) form on the GPU against the 3-D FP64 oracle: the filled matrix and field,
the dFOM of every pillar, greedy and top-k trajectories (complex128 within 1e-10, complex64
within the mixed-precision bounds), lock-step from the oracle's choices."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import gf_oracle3d as O3
from paper_2202_05388_gb300 import build as BLD
from paper_2202_05388_gb300 import gfopt as B
from paper_2202_05388_gb300 import workloads as W
from paper_2202_05388_gb300.optimizer import GreedyOptimizer3D

from gpu_parity import GAP, TOL, rel_err

C64_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BLD.build()


def _gpu_G(opt):
    return opt.G[:, :opt.n].cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("nx,ny,nz,dtype", [(4, 3, 2, "c128"), (5, 4, 3, "c128"), (4, 4, 2, "c64")])
def test_fill_matches_oracle(nx, ny, nz, dtype):
    g = W.small_3d(nx, ny, nz).geoms[0]
    opt = GreedyOptimizer3D(g, W.CandidateSpec(W.KIND_PILLAR, 3, 1), dtype=dtype)
    opt.fill()
    torch.cuda.synchronize()
    tol = 1e-12 if dtype == "c128" else 1e-7
    assert rel_err(_gpu_G(opt), O3.g0_matrix(g)) <= tol
    assert rel_err(opt.E.cpu().numpy(), O3.incident_field(g)) <= 1e-14
    assert abs(float(opt.fom.cpu()[0]) - O3.fom(O3.incident_field(g), g)) <= 1e-14


@pytest.mark.parametrize("nx,ny,nz,k,dtype,steps", [(4, 3, 2, 1, "c128", 6), (5, 5, 2, 1, "c128", 5),
                                                    (6, 5, 3, 2, "c128", 3), (5, 4, 2, 1, "c64", 5)])
def test_pillar_trajectory_lockstep_vs_oracle(nx, ny, nz, k, dtype, steps):
    wl = W.small_3d(nx, ny, nz, k=k)
    g = wl.geoms[0]
    spec = wl.spec
    opt = GreedyOptimizer3D(g, spec, dtype=dtype)
    opt.fill()
    orc = O3.OracleProblem3D(g, spec)
    tol = TOL if dtype == "c128" else C64_TOL
    done = 0
    for t in range(steps):
        opt.evaluate()
        d_orc = orc.evaluate()
        d_gpu = opt.dfom.cpu().numpy()
        fin = np.isfinite(d_orc)
        assert np.array_equal(fin, np.isfinite(d_gpu))
        scale = max(1.0, float(np.max(np.abs(d_orc[fin]))))
        assert np.max(np.abs(d_gpu[fin] - d_orc[fin])) <= (tol if dtype == "c128" else 1e-4) * scale, t
        ids = orc.choose(d_orc)
        if not ids:
            break
        opt.select()
        got = opt.read_step()
        if got.ids != ids:
            top = np.sort(d_orc[fin])[::-1]
            assert top[0] - top[1] <= GAP * abs(top[0]) or dtype == "c64", (t, got.ids, ids)
            fixed = torch.full((max(1, k),), -1, dtype=torch.int32)
            fixed[:len(ids)] = torch.tensor(ids, dtype=torch.int32)
            opt.idx.copy_(fixed.to(opt.idx.device))
            opt.status.zero_()
        orc.accept(ids)
        opt.update()
        torch.cuda.synchronize()
        assert int(opt.status.cpu()[0]) == B.GF_OK
        assert rel_err(_gpu_G(opt), orc.G) <= tol, t
        assert rel_err(opt.E.cpu().numpy(), orc.E) <= tol, t
        assert abs(float(opt.fom.cpu()[0]) - orc.fom()) <= tol * orc.fom(), t
        assert np.array_equal(opt.state.cpu().numpy(), orc.state), t
        done += 1
    assert done >= 2


def test_3d_validation():
    g = W.small_3d(4, 3, 2).geoms[0]
    h = B.Handle(0)
    spec = W.CandidateSpec(W.KIND_PILLAR, 3, 1)
    n = h.gf3_num_unknowns(g)
    assert n == 3 * (4 * 3 * 2 + 1)
    G = torch.empty((n, n + 1), dtype=torch.complex128, device="cuda")
    E = torch.empty(n, dtype=torch.complex128, device="cuda")
    ws = torch.empty(h.gf3_workspace_size(g, B.GF_C128, spec), dtype=torch.uint8, device="cuda")
    inside = W.Geometry3D(4, 3, 2, 0.05, 1.0, 0.1, 0.05, 0.05)
    with pytest.raises(B.GfError, match="inside the design slab"):
        h.gf3_fill_g0(B.problem3d_struct(inside, G, n + 1, E), B.GF_C128, ws, ws.numel())
    with pytest.raises(B.GfError, match="PILLAR"):
        h.gf3_eval_candidates(B.problem3d_struct(g, G, n + 1, E), B.GF_C128, torch.zeros(24, dtype=torch.uint8, device="cuda"),
                              W.CandidateSpec(W.KIND_BRUSH2, 3, 1), torch.empty(12, dtype=torch.float64, device="cuda"))
    with pytest.raises(B.GfError, match="ldg"):
        h.gf3_fill_g0(B.problem3d_struct(g, G, n - 1, E), B.GF_C128, ws, ws.numel())


def test_aligned_pillars_match_oracle():
    wl = W.small_3d(6, 5, 2)
    g = wl.geoms[0]
    spec = W.CandidateSpec(W.KIND_PILLAR, 3, 1, aligned=True)
    opt = GreedyOptimizer3D(g, spec, dtype="c128")
    opt.fill()
    orc = O3.OracleProblem3D(g, spec)
    for t in range(3):
        opt.evaluate()
        d_orc = orc.evaluate()
        d_gpu = opt.dfom.cpu().numpy()
        fin = np.isfinite(d_orc)
        assert np.array_equal(fin, np.isfinite(d_gpu))
        assert np.max(np.abs(d_gpu[fin] - d_orc[fin])) <= TOL * max(1.0, np.max(np.abs(d_orc[fin])))
        ids = orc.choose(d_orc)
        if not ids:
            break
        opt.select()
        orc.accept(ids)
        opt.update()
        torch.cuda.synchronize()
        assert np.array_equal(opt.state.cpu().numpy(), orc.state)


@pytest.mark.parametrize("nx,ny,nz,steps", [(24, 20, 4, 6), (17, 13, 2, 4)])
def test_c64_eval_fp32_factors_refined_match_fp64_factors(nx, ny, nz, steps):
    """Complex64 G: the pillar evaluation with FP32 factors and one FP64 refinement step
    (GF_UPDATE_TC) against FP64 factors of the same stored system (GF_UPDATE_DFMA), on every
    candidate after a few greedy steps: the refined solve reaches the FP64 solve of the stored
    matrix (both read the same FP32 entries), well inside the storage rounding of G."""
    wl = W.small_3d(nx, ny, nz, dtype="c64")
    opt = GreedyOptimizer3D(wl.geoms[0], wl.spec, dtype="c64")
    opt.fill()
    for _ in range(steps):
        opt.step()
    torch.cuda.synchronize()
    assert int(opt.status.cpu()[0]) == B.GF_OK
    opt.evaluate()
    d32 = opt.dfom.cpu().numpy().copy()
    opt.h.gf_set_update_algo(B.GF_UPDATE_DFMA)
    opt.evaluate()
    d64 = opt.dfom.cpu().numpy().copy()
    opt.h.gf_set_update_algo(B.GF_UPDATE_TC)
    fin = np.isfinite(d64)
    assert fin.sum() > 0.4 * fin.size
    assert np.array_equal(fin, np.isfinite(d32))
    scale = float(np.max(np.abs(d64[fin])))
    err = float(np.max(np.abs(d32[fin] - d64[fin])))
    print(f"max |dFOM(FP32 factors + refinement) - dFOM(FP64 factors)| = {err:.3e} (scale {scale:.3e})")
    assert err <= 1e-9 * scale
    assert int(np.argmax(np.where(fin, d32, -np.inf))) == int(np.argmax(np.where(fin, d64, -np.inf)))
