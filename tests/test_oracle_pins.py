"""Pins of the FP64 oracle against facts it does not compute itself (CPU only).

* G0 entries against mpmath's arbitrary-precision Hankel functions and the small-argument
  asymptotic form of H0 (independent special-function code).
* The pixel self term against adaptive quadrature of k^2 * int_disk (i/4) H0(k r) dA.
* Candidate dFOM against a brute-force re-solve of the full discrete Lippmann-Schwinger
  system of the flipped structure (Eqs. 2-3, Eq. 1).
* G and E after every accepted flip against brute-force solves (I - G0 X)^{-1} [G0, E_inc].
* Invariants: reciprocity G = G^T, E = E_inc + G X E_inc, order independence of flips,
  mirror symmetry of dFOM, monotone greedy FOM.
* Planted mistakes: each pin is shown to catch a plausible bug planted in the oracle.
"""
import math

import mpmath
import numpy as np
import pytest
from scipy.special import hankel1

from oracle import gf_oracle as O
from paper_2202_05388_gb300 import workloads as W

mpmath.mp.dps = 30


def _mp_h(order, x):
    return complex(mpmath.besselj(order, x) + 1j * mpmath.bessely(order, x))


def test_g0_pair_matches_mpmath():
    g = W.plain_32().geoms[0]
    k = 2 * math.pi / g.wavelength
    for r in [g.dx, math.sqrt(2) * g.dx, 3.7 * g.dx, 1.0, 2.9, 7.5]:
        ref = 0.25j * k * k * g.dx * g.dx * _mp_h(0, k * r)
        got = complex(O.g0_pair(g, r))
        assert abs(got - ref) <= 1e-14 * abs(ref), (r, got, ref)


def test_g0_small_argument_asymptote():
    # H0(x) = 1 + (2i/pi)(ln(x/2) + gamma) + O(x^2 ln x) as x -> 0
    g = W.plain_32().geoms[0]
    k = 2 * math.pi / g.wavelength
    r = 1e-7
    asym = 1 + (2j / math.pi) * (math.log(k * r / 2) + np.euler_gamma)
    got = complex(O.g0_pair(g, r)) / (0.25j * k * k * g.dx ** 2)
    assert abs(got - asym) < 1e-12


@pytest.mark.parametrize("ratio", [16, 20, 24])
def test_self_term_matches_disk_quadrature(ratio):
    # k^2 * int over a disk of area dx^2 of (i/4) H0(k r) dA = (i/4) k^2 2 pi int_0^a H0(k r) r dr
    g = W.small(4, 4, ratio=ratio).geoms[0]
    k = 2 * math.pi / g.wavelength
    a = g.dx / math.sqrt(math.pi)
    re = mpmath.quad(lambda r: r * mpmath.besselj(0, k * r), [0, a])
    im = mpmath.quad(lambda r: r * mpmath.bessely(0, k * r), [0, a / 1e6, a / 1e3, a])
    ref = 0.25j * k * k * 2 * math.pi * complex(re + 1j * im)
    got = O.g0_self(g)
    assert abs(got - ref) < 1e-13, (got, ref)


def test_g0_matrix_layout_and_reciprocity():
    g = W.small(5, 4).geoms[0]
    G = O.g0_matrix(g)
    assert G.shape == (g.n, g.n)
    assert np.array_equal(G, G.T)
    assert G[g.N, g.N] == 0
    # pixel (ix=1, iy=2) to pixel (ix=3, iy=0) is at distance sqrt(8) dx
    i, j = 2 * g.nx + 1, 0 * g.nx + 3
    assert abs(G[i, j] - O.g0_pair(g, math.sqrt(8) * g.dx)) == 0
    # monitor column uses the same off-diagonal rule
    pts = O.points(g)
    r = np.hypot(*(pts[g.N] - pts[7]))
    assert abs(G[7, g.N] - 0.25j * (2 * math.pi) ** 2 * g.dx ** 2 * _mp_h(0, 2 * math.pi * r)) < 1e-15


def test_gauss_pp_matches_lapack_and_flags_singular():
    rng = np.random.default_rng(1)
    for p in (1, 2, 4, 7):
        A = rng.normal(size=(p, p)) + 1j * rng.normal(size=(p, p))
        b = rng.normal(size=(p, 3)) + 1j * rng.normal(size=(p, 3))
        x, ok = O.gauss_pp(A, b)
        assert ok
        assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-12, atol=1e-12)
        xb, okb = O.gauss_pp_batch(np.stack([A, 2 * A]), np.stack([b[:, 0], b[:, 1]]))
        assert okb.all()
        assert np.allclose(xb[1], np.linalg.solve(2 * A, b[:, 1]), rtol=1e-12, atol=1e-12)
    S = np.array([[1.0, 2.0], [0.5, 1.0]], dtype=complex)
    assert not O.gauss_pp(S, np.ones(2))[1]
    assert not O.gauss_pp_batch(S[None], np.ones((1, 2)))[1][0]
    # an exactly zero matrix is singular (its relative threshold is zero too)
    Z = np.zeros((1, 1), dtype=complex)
    assert not O.gauss_pp(Z, np.ones(1))[1]
    assert not O.gauss_pp_batch(Z[None], np.ones((1, 1)))[1][0]


def _brute_dfom(g, state, V, d_sign):
    """FOM change from two full Lippmann-Schwinger solves."""
    s2 = state.copy()
    s2[V] ^= 1
    _, E0 = O.brute_force(g, state)
    _, E1 = O.brute_force(g, s2)
    return abs(E1[g.N]) ** 2 - abs(E0[g.N]) ** 2


@pytest.mark.parametrize("kind,dir_mask", [(W.KIND_SINGLE, W.DIR_FILL | W.DIR_CLEAR),
                                           (W.KIND_BRUSH2, W.DIR_FILL | W.DIR_CLEAR)])
def test_every_candidate_dfom_matches_brute_force(kind, dir_mask):
    wl = W.small(5, 4, kind=kind, dir_mask=dir_mask)
    g = wl.geoms[0]
    state = W.random_state(g.N, seed=3, fill=0.4)
    pr = O.OracleProblem(wl.geoms, wl.spec, state)
    dfom = pr.evaluate()
    nvalid = 0
    for cid in range(dfom.size):
        c = O.candidate(g, wl.spec, state, cid)
        if c is None:
            assert dfom[cid] == -np.inf
            continue
        nvalid += 1
        ref = _brute_dfom(g, state, c[0], None)
        assert abs(dfom[cid] - ref) <= 1e-11 * max(1.0, abs(ref)), (cid, dfom[cid], ref)
    assert nvalid > 0


def test_single_inclusion_from_vacuum():
    # From vacuum, one pixel j: E_m' = E_m + G0_mj chi E_inc_j / (1 - G0_jj chi)  (p = 1 Eq. 9)
    # checked here against the brute-force solve, and the oracle against both.
    g = W.small(4, 4).geoms[0]
    chi = g.eps_mat - g.eps_bg
    G0 = O.g0_matrix(g)
    Ei = O.incident_field(g)
    for j in (0, 5, 15):
        s = np.zeros(g.N, dtype=np.uint8)
        s[j] = 1
        _, Ebf = O.brute_force(g, s)
        closed = Ei[g.N] + G0[g.N, j] * chi * Ei[j] / (1 - G0[j, j] * chi)
        assert abs(Ebf[g.N] - closed) < 1e-14
    pr = O.OracleProblem([g], W.CandidateSpec())
    d = pr.evaluate()
    j = 5
    closed = Ei[g.N] + G0[g.N, j] * chi * Ei[j] / (1 - G0[j, j] * chi)
    assert abs(d[j] - (abs(closed) ** 2 - abs(Ei[g.N]) ** 2)) < 1e-14


def _check_against_brute(pr, tol=1e-12):
    for g, G, E in zip(pr.geoms, pr.Gs, pr.Es):
        Gb, Eb = O.brute_force(g, pr.state)
        assert np.max(np.abs(G - Gb)) <= tol * np.max(np.abs(Gb))
        assert np.max(np.abs(E - Eb)) <= tol * np.max(np.abs(Eb))


@pytest.mark.parametrize("wl,seed", [
    (W.small(6, 5, kind=W.KIND_SINGLE, dir_mask=W.DIR_FILL, steps=8), None),
    (W.small(6, 6, kind=W.KIND_SINGLE, dir_mask=W.DIR_FILL | W.DIR_CLEAR, steps=8), 11),
    (W.small(7, 6, kind=W.KIND_BRUSH2, dir_mask=W.DIR_FILL | W.DIR_CLEAR, steps=6), 12),
    (W.small(12, 10, kind=W.KIND_BRUSH2, dir_mask=W.DIR_FILL | W.DIR_CLEAR, k=3, excl_radius=3, steps=3), 13),
    (W.small(8, 4, kind=W.KIND_BRUSH2, dir_mask=W.DIR_FILL | W.DIR_CLEAR, wavelengths=(0.9, 1.0, 1.1),
             steps=4), 14),
], ids=["single_fill", "single_toggle", "brush", "brush_topk", "brush_multilambda"])
def test_trajectory_matches_brute_force_every_step(wl, seed):
    g = wl.geoms[0]
    state = None if seed is None else W.random_state(g.N, seed=seed, fill=0.3)
    pr = O.OracleProblem(wl.geoms, wl.spec, state)
    f_prev = pr.fom()
    taken = 0
    for _ in range(wl.steps):
        ids, dfom = pr.step()
        if not ids:
            break
        taken += 1
        f = pr.fom()
        assert f > f_prev                              # greedy FOM increases (Sec. IV)
        if len(ids) == 1:
            assert abs((f - f_prev) - dfom[ids[0]]) <= 1e-12 * max(1, f)
        f_prev = f
        _check_against_brute(pr)
        for G in pr.Gs:                                # reciprocity
            assert np.max(np.abs(G - G.T)) <= 1e-12 * np.max(np.abs(G))
    assert taken >= 2


def test_field_identity_e_equals_einc_plus_gxeinc():
    wl = W.small(6, 5, kind=W.KIND_BRUSH2, dir_mask=3, steps=4)
    pr = O.OracleProblem(wl.geoms, wl.spec, W.random_state(30, seed=4))
    for _ in range(wl.steps):
        pr.step()
    g = wl.geoms[0]
    x = np.zeros(g.n)
    x[:g.N] = pr.state * (g.eps_mat - g.eps_bg)
    Ei = O.incident_field(g)
    lhs = pr.Es[0]
    rhs = Ei + pr.Gs[0] @ (x * Ei)
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_flip_order_independence_and_joint_update():
    g = W.small(6, 6).geoms[0]
    chi = g.eps_mat - g.eps_bg
    G0, E0 = O.g0_matrix(g), O.incident_field(g)
    A, B = np.array([3, 4]), np.array([20, 27, 28])
    GA, EA, _ = O.apply_update(G0, E0, A, np.full(2, chi))
    GAB, EAB, _ = O.apply_update(GA, EA, B, np.full(3, chi))
    GB, EB, _ = O.apply_update(G0, E0, B, np.full(3, chi))
    GBA, EBA, _ = O.apply_update(GB, EB, A, np.full(2, chi))
    J = np.concatenate([A, B])
    GJ, EJ, _ = O.apply_update(G0, E0, J, np.full(5, chi))
    for X, Y in [(GAB, GBA), (GAB, GJ)]:
        assert np.max(np.abs(X - Y)) < 1e-14
    for X, Y in [(EAB, EBA), (EAB, EJ)]:
        assert np.max(np.abs(X - Y)) < 1e-13
    # flipping back restores the background exactly (up to rounding)
    Gr, Er, _ = O.apply_update(GJ, EJ, J, np.full(5, -chi))
    assert np.max(np.abs(Gr - G0)) < 1e-14 and np.max(np.abs(Er - E0)) < 1e-13


def test_mirror_symmetry_of_dfom():
    # geometry and incident wave are symmetric under ix -> nx-1-ix (monitor on the centre line)
    wl = W.small(8, 6, kind=W.KIND_SINGLE, dir_mask=W.DIR_FILL)
    g = wl.geoms[0]
    d = O.OracleProblem(wl.geoms, wl.spec).evaluate().reshape(g.ny, g.nx)
    assert np.max(np.abs(d - d[:, ::-1])) <= 1e-13 * np.max(np.abs(d))
    wb = W.small(8, 6, kind=W.KIND_BRUSH2, dir_mask=W.DIR_FILL)
    db = O.OracleProblem(wb.geoms, wb.spec).evaluate()[: 7 * 5].reshape(5, 7)
    assert np.max(np.abs(db - db[:, ::-1])) <= 1e-13 * np.max(np.abs(db))


def test_select_best_tie_rule():
    d = np.array([-1.0, 0.5, 2.0, 2.0 * (1 - 5e-13), 2.0, -np.inf])
    assert O.select_best(d, 1e-12) == 2
    d2 = np.array([1.0, 2.0 * (1 - 5e-13), 2.0])
    assert O.select_best(d2, 1e-12) == 1
    assert O.select_best(d2, 0.0) == 2
    assert O.select_best(np.array([-1.0, 0.0, -np.inf]), 1e-12) is None
    assert O.select_best(np.array([]), 1e-12) is None


def test_select_topk_properties():
    rng = np.random.default_rng(7)
    g = W.small(20, 18, kind=W.KIND_BRUSH2).geoms[0]
    spec = W.CandidateSpec(W.KIND_BRUSH2, 3, k=8, excl_radius=3)
    for trial in range(5):
        d = rng.normal(size=2 * 19 * 17)
        d[rng.random(d.size) < 0.2] = -np.inf
        t = O.select_topk(g, spec, d)
        assert len(t) <= 8 and len(set(t)) == len(t)
        anc = [O.anchor(g, spec, c) for c in t]
        for a in range(len(t)):
            assert d[t[a]] > 0
            for b in range(a):
                assert max(abs(anc[a][0] - anc[b][0]), abs(anc[a][1] - anc[b][1])) > 3
                assert (d[t[b]], -t[b]) > (d[t[a]], -t[a])
        # maximality: every positive candidate ranked above the last taken one conflicts
        last = (d[t[-1]], -t[-1])
        for c in range(d.size):
            if c in t or not d[c] > 0 or (d[c], -c) < last:
                continue
            ac = O.anchor(g, spec, c)
            assert any(max(abs(ac[0] - x[0]), abs(ac[1] - x[1])) <= 3 for x in anc)
        if len(t) < 8:   # ran out: every remaining positive candidate conflicts
            for c in range(d.size):
                if c not in t and d[c] > 0:
                    ac = O.anchor(g, spec, c)
                    assert any(max(abs(ac[0] - x[0]), abs(ac[1] - x[1])) <= 3 for x in anc)


def test_topk_joint_fallback_to_best_single():
    # a multi-candidate set is applied jointly only if its joint dFOM is positive
    wl = W.small(12, 10, kind=W.KIND_BRUSH2, dir_mask=3, k=4)
    g = wl.geoms[0]
    pr = O.OracleProblem(wl.geoms, wl.spec, W.random_state(g.N, seed=21, fill=0.3))
    d = pr.evaluate()
    ids = pr.choose(d)
    assert len(ids) >= 2
    V, dc = pr.flip_set(ids)
    joint = O.delta_fom(pr.Gs, pr.Es, V, dc)
    f0 = pr.fom()
    applied = pr.accept(ids)
    if joint > 0:
        assert applied == ids
        assert abs(pr.fom() - f0 - joint) < 1e-12 * max(1, f0)
    else:
        assert applied == ids[:1]


# ------------------------------------------------------------------ planted mistakes
def _planted(monkeypatch, name, fn):
    monkeypatch.setattr(O, name, fn)


def test_pins_catch_dropped_self_term_constant(monkeypatch):
    good = O.g0_self
    _planted(monkeypatch, "g0_self", lambda g: good(g) + 1.0)     # the "-1" dropped
    g = W.small(4, 4).geoms[0]
    k = 2 * math.pi / g.wavelength
    a = g.dx / math.sqrt(math.pi)
    re = mpmath.quad(lambda r: r * mpmath.besselj(0, k * r), [0, a])
    im = mpmath.quad(lambda r: r * mpmath.bessely(0, k * r), [0, a / 1e6, a / 1e3, a])
    ref = 0.25j * k * k * 2 * math.pi * complex(re + 1j * im)
    assert abs(O.g0_self(g) - ref) > 0.5


def test_pins_catch_wrong_update_sign_or_transpose(monkeypatch):
    # mixed fill/clear contrasts, so that G_VV D and D G_VV differ
    good = O.apply_update
    g = W.small(5, 4).geoms[0]
    chi = g.eps_mat - g.eps_bg
    s0 = np.zeros(g.N, dtype=np.uint8)
    s0[3] = 1
    G0, E0 = O.brute_force(g, s0)
    s1 = np.zeros(g.N, dtype=np.uint8)
    s1[9] = 1
    Gb, Eb = O.brute_force(g, s1)
    V, d = np.array([3, 9]), np.array([-chi, chi])
    Gn, En, _ = good(G0, E0, V, d)
    assert np.max(np.abs(Gn - Gb)) < 1e-12 and np.max(np.abs(En - Eb)) < 1e-12

    def wrong_sign(G, E, V, d):
        Gn, En, ok = good(G, E, V, d)
        return 2 * G - Gn, En, ok

    def transposed(G, E, V, d):
        A = np.eye(len(V)) - d[:, None] * G[np.ix_(V, V)]     # D G_VV instead of G_VV D
        R = np.linalg.solve(A, G[V, :])
        return G + G[:, V] @ (d[:, None] * R), E, True

    def no_monitor_coupling(G, E, V, d):
        Gn, En, ok = good(G, E, V, d)
        En = En.copy()
        En[-1] = E[-1]
        return Gn, En, ok

    for bad in (wrong_sign, transposed):
        Gx, _, _ = bad(G0, E0, V, d)
        assert np.max(np.abs(Gx - Gb)) > 1e-6
    _, Ex, _ = no_monitor_coupling(G0, E0, V, d)
    assert abs(Ex[-1] - Eb[-1]) > 1e-6


def test_pins_catch_wrong_dfom_index(monkeypatch):
    # dFOM built from the wrong row of G (a pixel row instead of the monitor row)
    wl = W.small(5, 4, kind=W.KIND_SINGLE, dir_mask=3)
    g = wl.geoms[0]
    state = W.random_state(g.N, seed=5)
    pr = O.OracleProblem(wl.geoms, wl.spec, state)
    bad = pr.Gs[0].copy()
    bad[g.N, :g.N] = bad[0, :g.N]
    d_bad = O.evaluate_all(wl.geoms, wl.spec, state, [bad], pr.Es)
    c = O.candidate(g, wl.spec, state, 7)
    ref = _brute_dfom(g, state, c[0], None)
    assert abs(d_bad[7] - ref) > 1e-6 * max(1, abs(ref))


def test_ls_residual_vanishes_for_exact_field_and_measures_a_perturbation():
    wl = W.small(7, 6)
    g = wl.geoms[0]
    state = W.random_state(g.N, seed=9, fill=0.4)
    _, E = O.brute_force(g, state)
    assert O.ls_residual(g, state, E) < 1e-14
    # perturb one pixel's field by delta: residual = ||delta e_j - G0 X delta e_j|| / ||E||
    j = int(np.flatnonzero(state)[0])
    delta = 1e-6
    E2 = E.copy()
    E2[j] += delta
    G0 = O.g0_matrix(g)
    x = np.zeros(g.n)
    x[:g.N] = state * (g.eps_mat - g.eps_bg)
    e = np.zeros(g.n, dtype=complex)
    e[j] = delta
    expect = np.linalg.norm(e - G0 @ (x * e)) / np.linalg.norm(E2)
    assert abs(O.ls_residual(g, state, E2) - expect) < 1e-12


def test_exact_columns_solve_the_dyson_system():
    g = W.small(5, 5).geoms[0]
    state = W.random_state(g.N, seed=10, fill=0.4)
    cols = [0, 7, g.N]
    C = O.exact_columns(g, state, cols)
    G0 = O.g0_matrix(g)
    x = np.zeros(g.n)
    x[:g.N] = state * (g.eps_mat - g.eps_bg)
    lhs = C - G0 @ (x[:, None] * C)
    assert np.max(np.abs(lhs - G0[:, cols])) < 1e-13


# --------------------------------------------------------------------------- epsilon-greedy (Sec. V)
def _ranked_improving(d):
    """Independent ranking: Python's tuple sort of (-dFOM, id) over the improving entries."""
    return [c for _, c in sorted((-float(v), c) for c, v in enumerate(d) if v > 0.0)]


def test_egreedy_exploit_branch_is_the_greedy_policy():
    rng = np.random.default_rng(41)
    for _ in range(100):
        d = rng.normal(size=40)
        d[rng.integers(0, 40, 3)] = d.max()          # exact ties at the maximum
        for u1 in (0.0, 0.3, 0.99):
            assert O.select_egreedy(d, 1e-12, 0.0, u1, rng.random()) == O.select_best(d, 1e-12)
        assert O.select_egreedy(d, 1e-12, 0.25, 0.25, rng.random()) == O.select_best(d, 1e-12)


def test_egreedy_explore_branch_picks_uniformly_among_the_top_four():
    rng = np.random.default_rng(42)
    for _ in range(100):
        d = np.round(rng.normal(size=30), 1)          # many exact ties below the top
        ranked = _ranked_improving(d)
        m = min(4, len(ranked))
        if m == 0:
            assert O.select_egreedy(d, 1e-12, 1.0, 0.0, 0.5) is None
            continue
        for r in range(m):
            for frac in (0.0, 0.5, 0.999):
                u2 = (r + frac) / m
                assert O.select_egreedy(d, 1e-12, 1.0, 0.0, u2) == ranked[r]


def test_egreedy_with_fewer_than_four_improving_and_none():
    d = np.array([-1.0, 0.5, -2.0, 0.25, 0.0, -0.1])
    assert [O.select_egreedy(d, 1e-12, 1.0, 0.1, u) for u in (0.0, 0.49, 0.5, 0.99)] == [1, 1, 3, 3]
    assert O.select_egreedy(-np.abs(d) - 1.0, 1e-12, 1.0, 0.0, 0.3) is None


def test_egreedy_choice_frequencies_match_the_closed_form():
    """On a midpoint grid of (u_explore, u_pick) the share of each rank is exactly
    (1 - eps) [r = 0] + eps / 4 (eps = 0.3, 40 x 40 grid, four improving candidates)."""
    d = np.array([0.9, 0.1, 0.4, -0.3, 0.7, 0.2, -1.0])
    ranked = _ranked_improving(d)[:4]                 # ids 0, 4, 2, 5
    grid = (np.arange(40) + 0.5) / 40
    counts = {c: 0 for c in ranked}
    for u1 in grid:
        for u2 in grid:
            counts[O.select_egreedy(d, 1e-12, 0.3, float(u1), float(u2))] += 1
    total = 40 * 40
    assert counts[ranked[0]] == round(total * (0.7 + 0.3 / 4))
    for c in ranked[1:]:
        assert counts[c] == round(total * 0.3 / 4)
