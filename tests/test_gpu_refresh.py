"""Drift refresh (gf_refresh) against the oracle's plain definitions: the Lippmann-Schwinger
residual of E (dense G0 X E) and exact columns of G ((I - G0 X)^{-1} G0).  Known perturbations
are injected into E and into one stored column on the device (host-side fault injection), so
the reported residuals are compared with values the oracle computes for the same data."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import gf_oracle as O
from paper_2202_05388_gb300 import build as BLD
from paper_2202_05388_gb300 import gfopt as B
from paper_2202_05388_gb300 import workloads as W
from paper_2202_05388_gb300.optimizer import GreedyOptimizer


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BLD.build()


def _prepare(nx, ny, seed, dtype):
    wl = W.small(nx, ny, kind=W.KIND_BRUSH2, dir_mask=3, dtype=dtype)
    g = wl.geoms[0]
    opt = GreedyOptimizer(wl.geoms, wl.spec, dtype=dtype)
    opt.fill()
    single = W.CandidateSpec(W.KIND_SINGLE, 3, 1)
    for j in np.flatnonzero(W.random_state(g.N, seed=seed, fill=0.3)):
        opt.force([int(j)], single)
    for _ in range(3):
        opt.step()
    torch.cuda.synchronize()
    return wl, g, opt


@pytest.mark.parametrize("nx,ny,dtype", [(12, 10, "c128"), (17, 9, "c128"), (16, 16, "c64")])
def test_refresh_reports_oracle_residuals(nx, ny, dtype):
    wl, g, opt = _prepare(nx, ny, 81, dtype)
    state = opt.state.cpu().numpy()
    cols = [0, g.N // 2 + 3, g.N]
    restart = 30
    ws_bytes = opt.h.gf_refresh_workspace_size(g, restart)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    # clean state: tiny residuals
    res, its, cres = opt.h.gf_refresh(opt.probs[0], opt.dtype, opt.state, cols, restart, 400, 1e-13, ws, ws_bytes)
    lim = 1e-11 if dtype == "c128" else 1e-5
    assert res[0] <= lim and max(res[1:]) <= lim, res
    assert max(cres) <= lim and min(cres) > 0.0, cres       # backward errors: small, never a tautological 0
    # inject: E[j] += dE, stored G[:, c] += dG (host-side edits of device data)
    j = int(np.flatnonzero(state)[0])
    dE, dG = 1e-6, 1e-6
    opt.E[0][j] += dE
    c = cols[1]
    opt.G[0][:, c] += dG
    torch.cuda.synchronize()
    E = opt.E[0].cpu().numpy()
    res, its, cres = opt.h.gf_refresh(opt.probs[0], opt.dtype, opt.state, cols, restart, 400, 1e-13, ws, ws_bytes)
    r_ref = O.ls_residual(g, state, E)
    assert abs(res[0] - r_ref) <= 1e-3 * r_ref + 1e-12, (res[0], r_ref)
    exact = O.exact_columns(g, state, cols)
    Gd = opt.G[0][:, :g.n].cpu().numpy().astype(np.complex128)
    for s, cc in enumerate(cols):
        drift = np.linalg.norm(Gd[:, cc] - exact[:, s]) / np.linalg.norm(exact[:, s])
        assert abs(res[1 + s] - drift) <= 1e-3 * drift + 1e-10, (s, res[1 + s], drift)
        assert its[s] < 400
    assert res[2] > 1e-7          # the perturbed column is flagged


@pytest.mark.parametrize("nx,ny,dtype", [(14, 12, "c128"), (16, 14, "c64")])
def test_scheduled_refresh_repairs_a_drifted_field(nx, ny, dtype):
    """Drift planted in E on the host (a relative perturbation of every entry) is caught by
    the field repair that GreedyOptimizer.run schedules every R steps: the Eq. 3 residual exceeds
    the stated tolerance, E is replaced by its GMRES solution and matches the oracle's field (the
    exact solve for the current design) again, and the FOM is rewritten from it."""
    from gpu_parity import gpu_E, rel_err, reach_state
    wl = W.small(nx, ny, kind=W.KIND_BRUSH2, dir_mask=3, dtype=dtype)
    g = wl.geoms[0]
    orc = O.OracleProblem(wl.geoms, wl.spec)
    opt = GreedyOptimizer(wl.geoms, wl.spec, dtype=dtype)
    opt.fill()
    reach_state(opt, orc, W.random_state(g.N, seed=91, fill=0.3))
    torch.cuda.synchronize()
    tol_e = 1e-10 if dtype == "c128" else 2e-5
    assert rel_err(gpu_E(opt), orc.Es[0]) <= tol_e
    # a clean field passes the check untouched
    rep = opt.refresh_fields()[0]
    assert not rep["e_replaced"] and rep["e_iters"] == 0 and rep["e_residual"] <= opt.E_TOL[opt.dtype]
    # plant drift above the repair tolerance: E <- E (1 + a w), w a fixed complex pattern of unit
    # modulus, a = 1e-6 (complex128 G; tolerance 1e-9) or 1e-4 (complex64 G; tolerance 1e-5)
    a = 1e-6 if dtype == "c128" else 1e-4
    w = torch.exp(1j * torch.arange(g.n, dtype=torch.float64, device="cuda") * 0.7)
    opt.E[0].mul_(1.0 + a * w)
    torch.cuda.synchronize()
    assert rel_err(gpu_E(opt), orc.Es[0]) > 0.5 * a
    # one greedy step with the refresh scheduled after it, the oracle taking the same choice
    res = opt.run(1, refresh_every=1)
    assert res[0].status == B.GF_OK
    orc.accept(res[0].ids)
    torch.cuda.synchronize()
    (step, reps, secs), = opt.refresh_log
    assert step == 1 and reps[0]["e_replaced"] and reps[0]["e_iters"] > 0
    assert reps[0]["e_residual"] > opt.E_TOL[opt.dtype] and reps[0]["e_residual_after"] <= 1e-12
    # the repaired field is the exact solve for the current design: the oracle's E (which the
    # oracle's own pins tie to the brute-force solve); complex64 storage does not enter the solve
    assert rel_err(gpu_E(opt), orc.Es[0]) <= 1e-10, rel_err(gpu_E(opt), orc.Es[0])
    assert abs(float(opt.fom.cpu()[0]) - orc.fom()) <= 1e-10 * orc.fom()
    assert abs(res[0].fom - orc.fom()) <= 1e-10 * orc.fom()
