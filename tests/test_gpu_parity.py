"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element,
on seeded synthetic inputs (relative error <= 1e-10 on G, E, FOM and dFOM; identical flip
sequence except where the oracle itself sees a near tie, then lock-step)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import gf_oracle as O
from paper_2202_05388_gb300 import build as BLD
from paper_2202_05388_gb300 import gfopt as B
from paper_2202_05388_gb300 import workloads as W
from paper_2202_05388_gb300.optimizer import GreedyOptimizer

from gpu_parity import (TOL, compare_dfom, compare_state, gpu_E, gpu_G, rel_err, run_parity)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BLD.build()


@pytest.mark.parametrize("nx,ny,ratio", [(1, 1, 20), (3, 1, 20), (7, 5, 16), (32, 32, 20), (17, 23, 24)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_fill_g0_matches_oracle(nx, ny, ratio, dtype):
    wl = W.small(nx, ny, ratio=ratio)
    g = wl.geoms[0]
    opt = GreedyOptimizer(wl.geoms, wl.spec, dtype=dtype)
    opt.fill()
    torch.cuda.synchronize()
    G0 = O.g0_matrix(g)
    Gg = gpu_G(opt)
    tol = 1e-12 if dtype == "c128" else 1e-7
    assert rel_err(Gg, G0) <= tol
    # padding columns are zero
    if opt.ldg > opt.n:
        assert torch.count_nonzero(opt.G[0][:, opt.n:]).item() == 0
    assert rel_err(gpu_E(opt), O.incident_field(g)) <= 1e-13
    bands = opt.bands[0].cpu().numpy().reshape(B.GF_NBANDS, -1)
    offs = [(0, 0), (1, 0), (-1, 0), (-1, 1), (1, -1), (0, 1), (0, -1), (1, 1), (-1, -1)]
    for b, (ddx, ddy) in enumerate(offs):
        for i in range(g.N):
            ix, iy = i % nx, i // nx
            jx, jy = ix + ddx, iy + ddy
            ref = G0[i, jy * nx + jx] if (0 <= jx < nx and 0 <= jy < ny) else 0.0
            assert abs(bands[b, i] - ref) <= tol * max(1e-300, np.max(np.abs(G0))), (b, i)


@pytest.mark.parametrize("kind,dir_mask,seed", [
    (W.KIND_SINGLE, W.DIR_FILL, None),
    (W.KIND_SINGLE, W.DIR_FILL | W.DIR_CLEAR, 5),
    (W.KIND_SINGLE, W.DIR_CLEAR, 6),
    (W.KIND_BRUSH2, W.DIR_FILL | W.DIR_CLEAR, 7),
    (W.KIND_BRUSH2, W.DIR_FILL, 8),
    (W.KIND_BRUSH2, W.DIR_CLEAR, 9),
])
def test_eval_candidates_matches_oracle(kind, dir_mask, seed):
    wl = W.small(13, 11, kind=kind, dir_mask=dir_mask)
    g = wl.geoms[0]
    state = None if seed is None else W.random_state(g.N, seed=seed, fill=0.35)
    orc = O.OracleProblem(wl.geoms, wl.spec, state)
    opt = GreedyOptimizer(wl.geoms, wl.spec)
    opt.fill()
    if state is not None:
        from gpu_parity import reach_state
        orc2 = O.OracleProblem(wl.geoms, wl.spec)
        reach_state(opt, orc2, state)
    opt.evaluate()
    torch.cuda.synchronize()
    compare_dfom(opt.dfom.cpu().numpy(), orc.evaluate())


@pytest.mark.parametrize("algo", [B.GF_UPDATE_TC, B.GF_UPDATE_TENSOR])
def test_plain_32x32_single_fill_100_steps(algo):
    """The 32x32 single-pixel workload in full: up to 100 greedy steps (the greedy run stops
    early when no fill improves the FOM; both sides must stop at the same step), G/E/FOM
    compared every 10 steps; with the default arithmetic (FP64 FMA at this size) and with the
    tensor-core update forced."""
    wl = W.plain_32()
    done, lock = run_parity(wl, wl.steps, check_every=10, algo=algo)
    assert done >= 50
    assert lock <= 10


@pytest.mark.parametrize("algo", [B.GF_UPDATE_TC, B.GF_UPDATE_TENSOR])
@pytest.mark.parametrize("nx,ny,seed,steps", [(12, 10, 21, 12), (9, 14, 22, 10)])
def test_brush_trajectory(nx, ny, seed, steps, algo):
    wl = W.small(nx, ny, kind=W.KIND_BRUSH2, dir_mask=3, steps=steps)
    state = W.random_state(nx * ny, seed=seed, fill=0.3)
    done, lock = run_parity(wl, steps, state=state, algo=algo)
    assert done >= 3


def test_single_toggle_trajectory_ragged():
    wl = W.small(19, 7, kind=W.KIND_SINGLE, dir_mask=3, steps=15)
    state = W.random_state(19 * 7, seed=23, fill=0.25)
    done, _ = run_parity(wl, 15, state=state)
    assert done >= 5


def test_topk_trajectory():
    wl = W.small(14, 12, kind=W.KIND_BRUSH2, dir_mask=3, k=3, excl_radius=3, steps=5)
    state = W.random_state(14 * 12, seed=24, fill=0.3)
    done, _ = run_parity(wl, 5, state=state)
    assert done >= 2


def test_top32_c128_trajectory():
    """Top-32 brushes in complex128: every joint capacitance system (a workspace for up to 128
    pixels) is factorised and solved in one cluster of CTAs, whose factors and row interchanges
    then give the FP64 panels."""
    wl = W.small(26, 22, kind=W.KIND_BRUSH2, dir_mask=3, k=32, excl_radius=2, steps=4)
    state = W.random_state(26 * 22, seed=27, fill=0.3)
    done, _ = run_parity(wl, 4, state=state)
    assert done >= 2


def test_multi_wavelength_trajectory():
    wl = W.small(10, 6, kind=W.KIND_BRUSH2, dir_mask=3, wavelengths=(0.9, 1.0, 1.1), steps=5)
    state = W.random_state(60, seed=25, fill=0.3)
    done, _ = run_parity(wl, 5, state=state)
    assert done >= 2


def test_multi_wavelength_topk_cluster_trajectory():
    """Three wavelengths, top-12 brushes (joint sets up to 48 pixels per wavelength): each
    wavelength's system is factorised and solved in its own cluster of CTAs, whose factors then
    give that wavelength's FP64 panels; lock-step with the oracle."""
    wl = W.small(20, 16, kind=W.KIND_BRUSH2, dir_mask=3, k=12, excl_radius=2, wavelengths=(0.9, 1.0, 1.1), steps=3)
    state = W.random_state(20 * 16, seed=28, fill=0.3)
    done, _ = run_parity(wl, 3, state=state)
    assert done >= 2


def test_no_improving_candidate_sets_status_and_changes_nothing():
    # From vacuum, no 2x2 brush of eps = 12.25 helps this small lens: the oracle stops at once.
    wl = W.small(12, 10, kind=W.KIND_BRUSH2, dir_mask=3)
    orc = O.OracleProblem(wl.geoms, wl.spec)
    assert orc.choose(orc.evaluate()) == []
    opt = GreedyOptimizer(wl.geoms, wl.spec)
    opt.fill()
    G_before = opt.G[0].clone()
    opt.step()
    r = opt.read_step()
    assert r.status == B.GF_ENOIMPROVE and r.ids == []
    assert torch.equal(opt.G[0], G_before)
    assert abs(r.fom - orc.fom()) <= 1e-15


def test_singular_capacitance_is_reported_not_applied():
    # Host-side fault injection: make 1 - G_jj d_chi = 0 exactly for pixel j by editing G on
    # the device (eps_mat = 9, so d_chi = 8 and G_jj = 1/8 are exact in FP64).
    import dataclasses
    wl0 = W.small(6, 5, kind=W.KIND_SINGLE, dir_mask=W.DIR_FILL)
    g = dataclasses.replace(wl0.geoms[0], eps_mat=9.0)
    wl = dataclasses.replace(wl0, geoms=(g,))
    opt = GreedyOptimizer(wl.geoms, wl.spec)
    opt.fill()
    j = 7
    chi = g.eps_mat - g.eps_bg
    opt.G[0][j, j] = complex(1.0 / chi, 0.0)
    opt.h.gf_extract_bands(opt.probs[0], opt.dtype, torch.cuda.current_stream())
    opt.evaluate()
    d = opt.dfom.cpu().numpy()
    assert d[j] == -math.inf and np.isfinite(np.delete(d, j)).all()
    G_before = opt.G[0].clone()
    opt.force([j])
    torch.cuda.synchronize()
    assert int(opt.status.cpu()[0]) == B.GF_ESINGULAR
    assert torch.equal(opt.G[0], G_before)
    assert opt.state.cpu().numpy()[j] == 0


@pytest.mark.parametrize("k,dtype,nlam", [(8, "c128", 1), (12, "c128", 1), (32, "c128", 1), (12, "c64", 1),
                                          (32, "c64", 1), (12, "c128", 3), (16, "c64", 3)])
def test_singular_joint_system_is_reported_not_applied(k, dtype, nlam):
    """Host-side fault injection into a joint set of k 2x2 brushes (p = 4k pixels): row j of
    A = I - G_VV D is made exactly zero (G[V_j, V_c] = 0 for c != j, G[V_j, V_j] = 1/d_chi with
    d_chi = 8), so A is singular whatever the pivot order.  p = 32 takes the one-CTA blocked
    solve, p = 48 and 128 the cluster solve (complex64: the resident-A update at 48, the
    streaming update at 128).  With several wavelengths only the middle one's system is made
    singular (each wavelength's system has its own cluster and flag).  Every CTA must see the
    same failed pivot, the status must read GF_ESINGULAR and every wavelength's G and E and the
    design must be unchanged."""
    import dataclasses
    nx = ny = 24
    wl0 = W.small(nx, ny, kind=W.KIND_BRUSH2, dir_mask=W.DIR_FILL, k=k, excl_radius=0,
                  wavelengths=(0.9, 1.0, 1.1)[:nlam] if nlam > 1 else (1.0,))
    wl = dataclasses.replace(wl0, geoms=tuple(dataclasses.replace(gg, eps_mat=9.0) for gg in wl0.geoms))
    g = wl.geoms[0]
    lb = nlam // 2                                          # the wavelength made singular
    opt = GreedyOptimizer(wl.geoms, wl.spec, dtype=dtype)
    opt.fill()
    torch.cuda.synchronize()
    # k disjoint brushes on even anchors, in a seeded order; V in the kernels' order
    rng = np.random.default_rng(40 + k)
    anchors = [(2 * a, 2 * b) for b in range((ny - 1) // 2) for a in range((nx - 1) // 2)]
    pick = rng.permutation(len(anchors))[:k]
    ids = [anchors[i][1] * (nx - 1) + anchors[i][0] for i in pick]
    state0 = np.zeros(g.N, dtype=np.uint8)
    V = np.concatenate([O.candidate(g, wl.spec, state0, cid)[0] for cid in ids])
    assert V.size == 4 * k and np.unique(V).size == V.size
    jv = int(V[V.size // 2 + 1])
    chi = g.eps_mat - g.eps_bg
    assert chi == 8.0
    Vt = torch.as_tensor(V, device=opt.G[lb].device)
    opt.G[lb][jv, Vt] = 0
    opt.G[lb][jv, jv] = complex(1.0 / chi, 0.0)
    torch.cuda.synchronize()
    G_before = [G.clone() for G in opt.G]
    E_before = [E.clone() for E in opt.E]
    opt.force(ids)
    torch.cuda.synchronize()
    assert int(opt.status.cpu()[0]) == B.GF_ESINGULAR
    for lam in range(nlam):
        assert torch.equal(opt.G[lam], G_before[lam])
        assert torch.equal(opt.E[lam], E_before[lam])
    assert not opt.state.cpu().numpy().any()
    # the library stays usable: the first brush alone (its 4 x 4 system does not hold row j)
    # is applied by the next call
    assert jv not in set(V[:4].tolist())
    opt.force([ids[0]])
    torch.cuda.synchronize()
    assert int(opt.status.cpu()[0]) == B.GF_OK
    assert int(opt.state.cpu().numpy().sum()) == 4


def test_host_validation_rejects_bad_arguments():
    wl = W.plain_32()
    opt = GreedyOptimizer(wl.geoms, wl.spec)
    g = wl.geoms[0]
    bad = B.problem_struct(g, opt.G[0], opt.n - 1, opt.E[0], opt.bands[0])      # ldg < n
    with pytest.raises(B.GfError) as e:
        opt.h.gf_fill_g0(bad, opt.dtype, opt.ws, opt.ws_bytes)
    assert e.value.status == B.GF_EINVAL and "ldg" in str(e.value)
    inside = W.with_monitor(g, 0.5, 0.5)
    p = B.problem_struct(inside, opt.G[0], opt.ldg, opt.E[0], opt.bands[0])
    with pytest.raises(B.GfError, match="inside the design region"):
        opt.h.gf_fill_g0(p, opt.dtype, opt.ws, opt.ws_bytes)
    with pytest.raises(B.GfError) as e:
        opt.h.gf_fill_g0(opt.probs[0], opt.dtype, opt.ws, 64)
    assert e.value.status == B.GF_ENOMEM
    with pytest.raises(B.GfError):
        opt.h.gf_select_topk(g, wl.spec, opt.dfom, opt.ncand + 1, opt.idx, opt.val, opt.status,
                             opt.ws, opt.ws_bytes)
    bad_spec = W.CandidateSpec(kind=5)
    with pytest.raises(B.GfError):
        opt.h.gf_eval_candidates(opt.probs, opt.dtype, opt.state, bad_spec, opt.dfom)
    # misaligned pointer
    off = B.problem_struct(g, opt.G[0].data_ptr() + 8, opt.ldg, opt.E[0], opt.bands[0])
    with pytest.raises(B.GfError, match="aligned"):
        opt.h.gf_extract_bands(off, opt.dtype)


@pytest.mark.parametrize("nx,ny", [(24, 20), (47, 33)])
def test_tensor_core_update_matches_dfma_update(nx, ny):
    """The tensor-core digit-product update and the native-DFMA update agree to ~1e-15 on
    ragged sizes (n not a multiple of the 128-row / 16-column tiles)."""
    wl = W.small(nx, ny, kind=W.KIND_BRUSH2, dir_mask=3)
    state = W.random_state(nx * ny, seed=31, fill=0.3)
    a = GreedyOptimizer(wl.geoms, wl.spec)
    b = GreedyOptimizer(wl.geoms, wl.spec)
    a.h.gf_set_update_algo(B.GF_UPDATE_TENSOR)        # the tensor-core form at any size
    b.h.gf_set_update_algo(B.GF_UPDATE_DFMA)
    a.fill()
    b.fill()
    single = W.CandidateSpec(W.KIND_SINGLE, 3, 1)
    for j in np.flatnonzero(state)[:40]:
        a.force([int(j)], single)
        b.force([int(j)], single)
    torch.cuda.synchronize()
    assert rel_err(gpu_G(a), gpu_G(b)) <= 1e-14
    for t in range(6):
        a.evaluate()
        a.select()
        b.idx.copy_(a.idx)
        b.status.copy_(a.status)
        a.update()
        b.update()
        torch.cuda.synchronize()
        e = rel_err(gpu_G(a), gpu_G(b))
        assert e <= 1e-14, (t, e)
        assert rel_err(gpu_E(a), gpu_E(b)) <= 1e-14
    assert int(a.status.cpu()[0]) in (B.GF_OK, B.GF_ENOIMPROVE)


@pytest.mark.parametrize("nx,ny,k,seed", [(60, 50, 8, 71), (90, 70, 32, 72), (40, 30, 16, 73)])
def test_pooled_topk_selection_matches_oracle(nx, ny, k, seed):
    """Top-k with exclusion on random dFOM arrays (pooled path and its exact fallback) against
    the oracle's sorted scan."""
    g = W.small(nx, ny, kind=W.KIND_BRUSH2).geoms[0]
    spec = W.CandidateSpec(W.KIND_BRUSH2, 3, k=k, excl_radius=3)
    h = B.Handle(0)
    nc = h.gf_num_candidates(g, spec)
    rng = np.random.default_rng(seed)
    ws_bytes = h.gf_workspace_size(g, 1, B.GF_C128, spec)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    for trial in range(4):
        d = rng.normal(size=nc)
        if trial == 1:
            d = -np.abs(d)                                  # nothing improves
        if trial == 2:
            d = np.round(d, 1)                              # many exact ties
        if trial == 3:
            d[rng.random(nc) < 0.97] = -np.inf              # sparse improving set
        dt = torch.tensor(d, dtype=torch.float64, device="cuda")
        idx = torch.full((k,), -7, dtype=torch.int32, device="cuda")
        val = torch.empty(k, dtype=torch.float64, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        h.gf_select_topk(g, spec, dt, nc, idx, val, st, ws, ws_bytes)
        torch.cuda.synchronize()
        ref = O.select_topk(g, spec, d)
        got = [int(x) for x in idx.cpu().numpy() if x >= 0]
        assert got == ref, (trial, got[:5], ref[:5])
        assert int(st.cpu()[0]) == (B.GF_OK if ref else B.GF_ENOIMPROVE)


@pytest.mark.parametrize("nx,ny,kind,seed", [(200, 200, W.KIND_SINGLE, 81), (193, 192, W.KIND_BRUSH2, 82)])
def test_greedy_selection_over_many_ctas_matches_oracle(nx, ny, kind, seed):
    """The greedy choice (k = 1) from 32768 candidates runs as a pass of many CTAs over chunks and
    a finishing CTA: against the oracle's select_best, and bit for bit against the one-CTA sweep
    (no workspace), on random arrays, arrays with nothing improving, exact ties of the maximum
    in several chunks, and a near tie (within tie_rel) in an earlier chunk than the maximum."""
    g = W.small(nx, ny, kind=kind).geoms[0]
    spec = W.CandidateSpec(kind, 3, k=1)
    h = B.Handle(0)
    nc = h.gf_num_candidates(g, spec)
    assert nc >= 32768
    rng = np.random.default_rng(seed)
    ws_bytes = h.gf_workspace_size(g, 1, B.GF_C128, spec)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    chunk = -(-nc // 148)
    for trial in range(6):
        d = rng.normal(size=nc)
        if trial == 1:
            d = -np.abs(d)                                  # nothing improves
        if trial == 2:
            d[[nc - 5, 7 * chunk + 3, 2 * chunk - 1, 40 * chunk]] = 10.0      # exact ties of the max
        if trial == 3:
            d[nc - 1] = 10.0
            d[3 * chunk] = 10.0 * (1.0 - 0.25 * spec.tie_rel)               # within tie_rel, earlier
            d[chunk - 1] = 10.0 * (1.0 - 4.0 * spec.tie_rel)                # outside it
        if trial == 4:
            d[rng.random(nc) < 0.999] = -np.inf             # sparse improving set
        if trial == 5:
            d[rng.random(nc) < 0.01] = np.nan               # NaN never wins (GPU paths only)
        out = []
        for w in (ws, None):
            dt = torch.tensor(d, dtype=torch.float64, device="cuda")
            idx = torch.full((1,), -7, dtype=torch.int32, device="cuda")
            val = torch.empty(1, dtype=torch.float64, device="cuda")
            st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
            h.gf_select_topk(g, spec, dt, nc, idx, val, st, w, ws_bytes if w is not None else 0)
            torch.cuda.synchronize()
            out.append((int(idx.cpu()[0]), float(val.cpu()[0]), int(st.cpu()[0])))
        assert out[0][0] == out[1][0] and out[0][2] == out[1][2], (trial, out)
        assert np.array_equal(np.float64(out[0][1]), np.float64(out[1][1])), (trial, out)
        if trial == 5:
            ref = O.select_best(np.where(np.isnan(d), -np.inf, d), spec.tie_rel)
        else:
            ref = O.select_best(d, spec.tie_rel)
        got, v, s = out[0]
        if ref is None:
            assert s == B.GF_ENOIMPROVE and got == -1, (trial, out)
        else:
            assert s == B.GF_OK and got == ref and v == d[ref], (trial, got, ref)
        if trial == 2:
            assert got == 2 * chunk - 1
        if trial == 3:
            assert got == 3 * chunk


def test_bounded_wait_reports_timeout_and_context_survives():
    """A wait that nothing satisfies gives up after its limit and reports GF_ETIMEOUT through the
    device status word (no fault); the next greedy step on the same context is unaffected."""
    import time
    wl = W.plain_32()
    opt = GreedyOptimizer(wl.geoms, wl.spec)
    opt.fill()
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    opt.h.gf_selftest_timeout(50_000_000, st)            # 50 ms
    torch.cuda.synchronize()
    assert int(st.cpu()[0]) == B.GF_ETIMEOUT
    assert time.perf_counter() - t0 >= 0.045
    r = opt.run(3)
    assert r[0].status == B.GF_OK and len(r[0].ids) == 1
    with pytest.raises(B.GfError):
        opt.h.gf_selftest_timeout(10, st)


def test_topk_grid_barrier_timeout_reports_status_and_context_survives():
    """The one-launch top-k's grid barrier waits for one CTA more than its grid holds: every
    CTA's bounded wait gives up, the status word reports GF_ETIMEOUT (no fault), and a top-32
    selection on the same context afterwards matches the oracle."""
    import time
    h = B.Handle(0)
    nb = h.gf_select_selftest_bytes()
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    h.gf_select_selftest_timeout(50_000_000, ws, nb, st)    # 50 ms
    torch.cuda.synchronize()
    assert int(st.cpu()[0]) == B.GF_ETIMEOUT
    assert time.perf_counter() - t0 >= 0.045
    with pytest.raises(B.GfError):
        h.gf_select_selftest_timeout(50_000_000, ws, nb - 8, st)
    g = W.small(90, 70, kind=W.KIND_BRUSH2).geoms[0]
    spec = W.CandidateSpec(W.KIND_BRUSH2, 3, k=32, excl_radius=3)
    nc = h.gf_num_candidates(g, spec)
    d = np.random.default_rng(5).normal(size=nc)
    wsb = h.gf_workspace_size(g, 1, B.GF_C128, spec)
    wsel = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    idx = torch.full((32,), -7, dtype=torch.int32, device="cuda")
    val = torch.empty(32, dtype=torch.float64, device="cuda")
    h.gf_select_topk(g, spec, torch.tensor(d, device="cuda"), nc, idx, val, st, wsel, wsb)
    torch.cuda.synchronize()
    assert [int(x) for x in idx.cpu().numpy() if x >= 0] == O.select_topk(g, spec, d)
    assert int(st.cpu()[0]) == B.GF_OK
