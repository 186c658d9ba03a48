"""Pins of the 3-D (dyadic) FP64 oracle against facts it does not compute itself (CPU only).

* The dyadic block against mpmath's numerical second derivatives of the scalar Green's
  function: G0 = (I + grad grad / k^2) e^{ikR} / (4 pi R).
* The voxel self block against quadrature of that dyadic over the equal-volume sphere.
* Every pillar's dFOM, and G and E after every flip, against brute-force solves of the full
  3n x 3n system (I - G0 X) [G, E] = [G0, E_inc].
* Invariants: reciprocity G = G^T, mirror symmetry of the on-axis focus problem, the far-field
  transversality of G0.  A planted mistake (dropped R^R^ term) is caught.
"""
import math

import mpmath
import numpy as np
import pytest

from oracle import gf_oracle as O
from oracle import gf_oracle3d as O3
from paper_2202_05388_gb300 import workloads as W

mpmath.mp.dps = 30


def _geom(nx=3, ny=3, nz=2, focus=1.0):
    return W.small_3d(nx, ny, nz, focus=focus).geoms[0]


def test_dyadic_matches_mpmath_hessian_of_the_scalar_green_function():
    g = _geom()
    k = O3.wavenumber(g)
    dV = g.dx ** 3
    rng = np.random.default_rng(3)
    for _ in range(6):
        R = rng.normal(size=3) * rng.uniform(0.05, 2.0)
        got = O3.dyadic(g, R[None, :])[0] / (k * k * dV)

        def gs(x, y, z):
            r = mpmath.sqrt(x * x + y * y + z * z)
            return mpmath.exp(1j * k * r) / (4 * mpmath.pi * r)

        want = np.zeros((3, 3), dtype=np.complex128)
        for a in range(3):
            for b in range(3):
                order = [0, 0, 0]
                order[a] += 1
                order[b] += 1
                h = complex(mpmath.diff(gs, tuple(float(v) for v in R), tuple(order)))
                want[a, b] = (complex(gs(*[float(v) for v in R])) if a == b else 0.0) + h / (k * k)
        assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))


def test_self_block_matches_quadrature_of_the_dyadic_over_the_sphere():
    """k^2 int_{delta < r < a} G0 dV (Gauss-Legendre in r, theta, phi) + the analytic
    O(delta^2) core equals self_term + 1/3 (the depolarisation removed) times I."""
    g = _geom()
    k = O3.wavenumber(g)
    dV = g.dx ** 3
    a = (3.0 * dV / (4.0 * math.pi)) ** (1.0 / 3.0)
    delta = 1e-3 * a
    xr, wr = np.polynomial.legendre.leggauss(40)
    xt, wt = np.polynomial.legendre.leggauss(24)
    xp, wp = np.polynomial.legendre.leggauss(24)
    r = delta + (a - delta) * (xr + 1) / 2
    wr = wr * (a - delta) / 2
    th = math.pi * (xt + 1) / 2
    wt = wt * math.pi / 2
    ph = math.pi * (xp + 1)
    wp = wp * math.pi
    Rr, Tt, Pp = np.meshgrid(r, th, ph, indexing="ij")
    W3 = wr[:, None, None] * wt[None, :, None] * wp[None, None, :] * Rr ** 2 * np.sin(Tt)
    R = np.stack([Rr * np.sin(Tt) * np.cos(Pp), Rr * np.sin(Tt) * np.sin(Pp), Rr * np.cos(Tt)], axis=-1)
    D = O3.dyadic(g, R.reshape(-1, 3)).reshape(R.shape[:3] + (3, 3)) / dV      # k^2 G0
    integral = np.einsum("ijk,ijkab->ab", W3, D)
    core = (2.0 / 3.0) * (k * delta) ** 2 / 2.0      # k^2 int_0^delta (2/3) r e^{ikr} dr, leading order
    want = (O3.self_term(g) + 1.0 / 3.0 - core) * np.eye(3)
    assert np.max(np.abs(integral - want)) <= 1e-8


def test_far_field_is_transverse():
    g = _geom()
    k = O3.wavenumber(g)
    u = np.array([0.3, -0.5, 0.81])
    u /= np.linalg.norm(u)
    errs = []
    for kr in (50.0, 500.0):
        R = u * kr / k
        D = O3.dyadic(g, R[None, :])[0]
        far = (D[0, 0] / (1.0 + (1j * kr - 1) / kr ** 2 + (3 - 3j * kr - kr ** 2) / kr ** 2 * u[0] ** 2)) * (np.eye(3) - np.outer(u, u))
        errs.append(np.max(np.abs(D - far)) / np.max(np.abs(D)))
    assert errs[1] < errs[0] / 5 and errs[1] < 1e-2


def test_every_pillar_dfom_matches_brute_force():
    g = _geom(3, 3, 2)
    spec = W.CandidateSpec(W.KIND_PILLAR, 3, 1)
    state = np.zeros(g.N, dtype=np.uint8)
    state[[1, 4, 10]] = 1
    G, E = O3.brute_force(g, state)
    f0 = O3.fom(E, g)
    d = O3.evaluate_all(g, spec, state, G, E)
    for c in range(d.size):
        V, dc = O3.candidate(g, spec, state, c)
        if V.size == 0:
            assert d[c] == -np.inf
            continue
        new = state.copy()
        new[np.unique(V // 3)] ^= 1
        _, E2 = O3.brute_force(g, new)
        assert abs(d[c] - (O3.fom(E2, g) - f0)) <= 1e-11 * max(1.0, f0)


def test_greedy_pillar_trajectory_matches_brute_force_and_is_reciprocal():
    g = _geom(4, 3, 2)
    orc = O3.OracleProblem3D(g, W.CandidateSpec(W.KIND_PILLAR, 3, 1))
    prev = orc.fom()
    for _ in range(5):
        ids, _ = orc.step()
        if not ids:
            break
        Gb, Eb = O3.brute_force(g, orc.state)
        assert np.max(np.abs(orc.G - Gb)) <= 1e-12 * np.max(np.abs(Gb))
        assert np.max(np.abs(orc.E - Eb)) <= 1e-12 * np.max(np.abs(Eb))
        assert np.max(np.abs(orc.G - orc.G.T)) <= 1e-12 * np.max(np.abs(orc.G))
        assert orc.fom() > prev
        prev = orc.fom()


def test_mirror_symmetric_pillars_have_equal_dfom():
    g = _geom(5, 3, 2)              # focus on the axis x = nx dx / 2: mirror x -> nx dx - x
    spec = W.CandidateSpec(W.KIND_PILLAR, 3, 1)
    state = np.zeros(g.N, dtype=np.uint8)
    G, E = O3.g0_matrix(g), O3.incident_field(g)
    d = O3.evaluate_all(g, spec, state, G, E)
    P = (g.nx - 1) * (g.ny - 1)
    for a in range(P):
        ay, ax = divmod(a, g.nx - 1)
        m = ay * (g.nx - 1) + (g.nx - 2 - ax)
        assert abs(d[a] - d[m]) <= 1e-12 * max(1e-30, abs(d[a]))


def test_pins_catch_a_dropped_rr_term(monkeypatch):
    g = _geom()
    orig = O3.dyadic

    def planted(gg, R):
        k = O3.wavenumber(gg)
        r = np.linalg.norm(R, axis=-1)
        kr = k * r
        A = 1.0 + (1j * kr - 1.0) / kr ** 2
        ph = np.exp(1j * kr) / (4 * math.pi * r)
        return (k * k * gg.dx ** 3) * (ph * A)[..., None, None] * np.eye(3)

    monkeypatch.setattr(O3, "dyadic", planted)
    with pytest.raises(AssertionError):
        test_dyadic_matches_mpmath_hessian_of_the_scalar_green_function()
    monkeypatch.setattr(O3, "dyadic", orig)


def test_aligned_candidates_are_the_even_partitions():
    g = _geom(5, 5, 2)
    spec = W.CandidateSpec(W.KIND_PILLAR, 3, 1, aligned=True)
    state = np.zeros(g.N, dtype=np.uint8)
    valid = [c for c in range(O3.num_candidates(g, spec)) if O3.candidate(g, spec, state, c)[0].size]
    P = (g.nx - 1) * (g.ny - 1)
    want = [c for c in range(P) if (c % (g.nx - 1)) % 2 == 0 and (c // (g.nx - 1)) % 2 == 0]   # fill only (vacuum)
    assert valid == want
