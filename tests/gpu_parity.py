"""Helpers for the GPU-vs-oracle parity tests (imported by tests/test_gpu_*.py only)."""
import numpy as np
import torch

from oracle import gf_oracle as O
from paper_2202_05388_gb300 import gfopt as B
from paper_2202_05388_gb300 import workloads as W
from paper_2202_05388_gb300.optimizer import GreedyOptimizer

TOL = 1e-10          # relative error bound on G, E, FOM and dFOM (max-norm relative)
GAP = 1e-9           # top-two dFOM gap below which the choice is a near tie


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def gpu_G(opt, l=0):
    return opt.G[l][:, :opt.n].cpu().numpy().astype(np.complex128)


def gpu_E(opt, l=0):
    return opt.E[l].cpu().numpy()


def reach_state(opt, orc, state):
    """Flip pixels one at a time (forced single-pixel toggles) on both sides."""
    single = W.CandidateSpec(W.KIND_SINGLE, W.DIR_FILL | W.DIR_CLEAR, 1)
    for j in np.flatnonzero(state):
        opt.force([int(j)], single)
        V, d = O.candidate(orc.geoms[0], single, orc.state, int(j))
        newG, newE = [], []
        for G, E in zip(orc.Gs, orc.Es):
            Gn, En, ok = O.apply_update(G, E, V, d)
            assert ok
            newG.append(Gn)
            newE.append(En)
        orc.Gs, orc.Es = newG, newE
        orc.state[V] ^= 1


def compare_state(opt, orc, tol=TOL, tag=""):
    for l in range(len(orc.geoms)):
        eG = rel_err(gpu_G(opt, l), orc.Gs[l])
        eE = rel_err(gpu_E(opt, l), orc.Es[l])
        assert eG <= tol, f"{tag} G rel err {eG:.3e} (wavelength {l})"
        assert eE <= tol, f"{tag} E rel err {eE:.3e} (wavelength {l})"
        bands = opt.bands[l].cpu().numpy().reshape(B.GF_NBANDS, -1)
        assert rel_err(bands[0], np.diag(orc.Gs[l])[:-1]) <= tol
    assert np.array_equal(opt.state.cpu().numpy(), orc.state), f"{tag} state differs"


def compare_dfom(d_gpu, d_orc, tag=""):
    fin = np.isfinite(d_orc)
    assert np.array_equal(fin, np.isfinite(d_gpu)), f"{tag} invalid-candidate sets differ"
    if fin.any():
        scale = max(1.0, float(np.max(np.abs(d_orc[fin]))))
        err = float(np.max(np.abs(d_gpu[fin] - d_orc[fin]))) / scale
        assert err <= TOL, f"{tag} dFOM err {err:.3e}"


def near_tie(d, chosen):
    """True when another candidate's dFOM is within GAP (relative) of the chosen maximum."""
    m = d[chosen[0]]
    others = np.delete(d, chosen)
    others = others[np.isfinite(others)]
    return others.size > 0 and np.max(others) >= m - GAP * abs(m)


def run_parity(wl, steps, state=None, check_every=1, dtype="c128", compare_every_G=True, algo=None):
    """Advance the GPU path and the oracle side by side; returns (n_steps, n_lockstep).
    algo: the update arithmetic (gf_set_update_algo), the library default when None."""
    orc = O.OracleProblem(wl.geoms, wl.spec)
    opt = GreedyOptimizer(wl.geoms, wl.spec, dtype=dtype)
    if algo is not None:
        opt.h.gf_set_update_algo(algo)
    opt.fill()
    torch.cuda.synchronize()
    compare_state(opt, orc, tag="fill")
    if state is not None and state.any():
        reach_state(opt, orc, state)
        torch.cuda.synchronize()
        compare_state(opt, orc, tag="initial state")
    lock = 0
    done = 0
    for t in range(steps):
        opt.evaluate()
        d_orc = orc.evaluate()
        d_gpu = opt.dfom.cpu().numpy()
        compare_dfom(d_gpu, d_orc, tag=f"step {t}")
        ids_orc = orc.choose(d_orc)
        opt.select()
        r = opt.read_step()
        if not ids_orc:
            assert r.status == B.GF_ENOIMPROVE, f"step {t}: oracle found no improving candidate"
            fom_before = float(opt.fom.cpu()[0])
            opt.update()          # must be a no-op
            torch.cuda.synchronize()
            compare_state(opt, orc, tag=f"step {t} no-op")
            break
        assert r.status == B.GF_OK
        if r.ids != ids_orc:
            # allowed only where the oracle itself sees a near tie
            assert len(r.ids) == len(ids_orc), f"step {t}: {r.ids} vs {ids_orc}"
            for a, b in zip(r.ids, ids_orc):
                assert abs(d_orc[a] - d_orc[b]) <= GAP * abs(d_orc[b]), \
                    f"step {t}: GPU chose {r.ids}, oracle {ids_orc} without a near tie"
            k = max(1, wl.spec.k)
            fixed = torch.full((k,), -1, dtype=torch.int32)
            fixed[:len(ids_orc)] = torch.tensor(ids_orc, dtype=torch.int32)
            opt.idx.copy_(fixed.to(opt.idx.device))
            lock += 1
        opt.update()
        orc.accept(ids_orc)
        done += 1
        torch.cuda.synchronize()
        f_gpu = float(opt.fom.cpu()[0])
        f_orc = orc.fom()
        assert abs(f_gpu - f_orc) <= TOL * abs(f_orc), f"step {t}: FOM {f_gpu} vs {f_orc}"
        if compare_every_G and ((t + 1) % check_every == 0 or t == steps - 1):
            compare_state(opt, orc, tag=f"step {t}")
    return done, lock
