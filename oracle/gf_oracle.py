"""Plain FP64 CPU oracle of the Green's-function pixel-by-pixel optimizer.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this module.
The CUDA product path never imports, links or calls it, and it imports nothing from the
product path except the input records in ``paper_2202_05388_gb300.workloads``.

What it computes (Wang et al., arXiv:2202.05388), restated for the 2-D scalar E_z problem:

* Background Green's matrix G0 over the n = N+1 points (N pixels, monitor last),
  with the paper's b = k0^2 * d_eps * dV folded into G so that b becomes the per-pixel
  contrast change d_chi (Sec. II, Eq. 4 and the "initial G known analytically" remark of
  Sec. II-B / Sec. IV):
      G_ij = (i/4) k^2 dx^2 H0(k |r_i - r_j|)          i != j (monitor row/column too)
      G_jj = (i pi/2) k a H1(k a) - 1,  a = dx/sqrt(pi) (pixel self term: the exact
             integral of k^2 (i/4) H0 over a disk of the pixel's area)
      G_NN = 0 (never read)
* Incident field E_inc(r) = exp(i k y).
* Candidate evaluation (Sec. II-A, Eqs. 4-9 and the partition form of Sec. III):
      A = I - G_VV D,  y = A^{-1} E_V,  E_m' = E_m + sum_i G_{m,i} d_chi_i y_i,
      dFOM = |E_m'|^2 - |E_m|^2                          (FOM of Eq. 1 = |E_m|^2)
* Update after a selection (Sec. II-B, Eqs. 10-14 and Eq. 4):
      R = A^{-1} G[V, :]   (Eq. 14),   G <- G + G[:, V] D R   (Eq. 10),
      E <- E + G[:, V] D y  (Eq. 4 with the new E_V of Eq. 9).
* Greedy selection (Fig. 1, Sec. III reduction): the maximum dFOM; stop when no
  candidate improves the FOM (Sec. IV).  Ties go to the lowest candidate id within a
  relative window tie_rel of the maximum.
* Top-k variant: candidates ordered by (-dFOM, id), taken greedily while they do not
  conflict (Chebyshev anchor distance <= excl_radius) with a taken one; the union is
  applied as one joint update when its joint dFOM is positive, else only the best one.
* epsilon-greedy policy (Sec. V): with probability 1 - epsilon the greedy choice, with
  probability epsilon a uniformly random one of the (up to) four best improving
  candidates ranked by (-dFOM, id).  The two uniform numbers of a step are inputs.
* Brute force (discrete Eqs. 2-3): G = (I - G0 X)^{-1} G0 and E = (I - G0 X)^{-1} E_inc.

Everything is complex128 / float64 with numpy and scipy.special.hankel1 as the only
library primitives (plus numpy.linalg.solve in the brute force).
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence, Tuple

import numpy as np
from scipy.special import hankel1

from paper_2202_05388_gb300.workloads import (CandidateSpec, Geometry, KIND_SINGLE, KIND_BRUSH2,
                                              DIR_FILL, DIR_CLEAR)

SINGULAR_REL = 1e-13   # |pivot| below this times ||A||_inf marks a candidate invalid


# --------------------------------------------------------------------------- geometry
def wavenumber(g: Geometry) -> float:
    """k = 2 pi / lambda in the (vacuum) background (Sec. II)."""
    return 2.0 * math.pi / g.wavelength


def points(g: Geometry) -> np.ndarray:
    """(n, 2) coordinates: pixel centres in row-major order, then the monitor."""
    ix = np.arange(g.nx, dtype=np.float64)
    iy = np.arange(g.ny, dtype=np.float64)
    X, Y = np.meshgrid((ix + 0.5) * g.dx, (iy + 0.5) * g.dx)   # Y rows, X columns
    pts = np.empty((g.N + 1, 2))
    pts[:g.N, 0] = X.ravel()
    pts[:g.N, 1] = Y.ravel()
    pts[g.N] = (g.mon_x, g.mon_y)
    return pts


def incident_field(g: Geometry) -> np.ndarray:
    """E_inc(r) = exp(i k y) at every point (plane wave along +y)."""
    return np.exp(1j * wavenumber(g) * points(g)[:, 1])


def contrast(g: Geometry) -> float:
    """chi of the patterning material relative to the background."""
    return g.eps_mat - g.eps_bg


# --------------------------------------------------------------------------- G0
def g0_pair(g: Geometry, r) -> np.ndarray:
    """(i/4) k^2 dx^2 H0^(1)(k r): the 2-D scalar Green's function integrated by the
    point rule over a pixel of area dx^2, with k^2 folded in."""
    k = wavenumber(g)
    return 0.25j * k * k * g.dx * g.dx * hankel1(0, k * np.asarray(r, dtype=np.float64))


def g0_self(g: Geometry) -> complex:
    """k^2 times the integral of (i/4) H0(k r) over a disk of area dx^2:
    (i pi / 2) k a H1(k a) - 1 with a = dx / sqrt(pi)."""
    k = wavenumber(g)
    a = g.dx / math.sqrt(math.pi)
    return complex(0.5j * math.pi * k * a * hankel1(1, k * a) - 1.0)


def g0_matrix(g: Geometry) -> np.ndarray:
    """Dense background Green's matrix over the n = N+1 points."""
    pts = points(g)
    d = pts[:, None, :] - pts[None, :, :]
    r = np.sqrt(d[..., 0] ** 2 + d[..., 1] ** 2)
    n = g.N + 1
    off = ~np.eye(n, dtype=bool)
    G = np.zeros((n, n), dtype=np.complex128)
    G[off] = g0_pair(g, r[off])
    idx = np.arange(g.N)
    G[idx, idx] = g0_self(g)
    G[g.N, g.N] = 0.0
    return G


# --------------------------------------------------------------------------- candidates
def num_candidates(g: Geometry, spec: CandidateSpec) -> int:
    if spec.kind == KIND_SINGLE:
        return g.N
    return 2 * (g.nx - 1) * (g.ny - 1)


def candidate(g: Geometry, spec: CandidateSpec, state: np.ndarray, cid: int
              ) -> Optional[Tuple[np.ndarray, np.ndarray]]:
    """Flipped pixel set V and its contrast changes for candidate ``cid``; None when the
    candidate changes nothing or its direction is not enabled."""
    chi = contrast(g)
    if spec.kind == KIND_SINGLE:
        j = cid
        if state[j] == 0 and spec.dir_mask & DIR_FILL:
            return np.array([j]), np.array([chi])
        if state[j] == 1 and spec.dir_mask & DIR_CLEAR:
            return np.array([j]), np.array([-chi])
        return None
    P = (g.nx - 1) * (g.ny - 1)
    direction, a = divmod(cid, P)
    if not spec.dir_mask & (DIR_FILL if direction == 0 else DIR_CLEAR):
        return None
    ax, ay = a % (g.nx - 1), a // (g.nx - 1)
    if getattr(spec, "aligned", False) and (ax % 2 or ay % 2):
        return None                                  # Sec. IV: aligned 2x2 partitions only
    j0 = ay * g.nx + ax
    brush = [j0, j0 + 1, j0 + g.nx, j0 + g.nx + 1]
    want_from = 0 if direction == 0 else 1          # only pixels that actually change
    V = np.array([j for j in brush if state[j] == want_from], dtype=np.int64)
    if V.size == 0:
        return None
    return V, np.full(V.size, chi if direction == 0 else -chi)


def anchor(g: Geometry, spec: CandidateSpec, cid: int) -> Tuple[int, int]:
    if spec.kind == KIND_SINGLE:
        return cid % g.nx, cid // g.nx
    a = cid % ((g.nx - 1) * (g.ny - 1))
    return a % (g.nx - 1), a // (g.nx - 1)


# --------------------------------------------------------------------------- small solves
def gauss_pp(A: np.ndarray, B: np.ndarray) -> Tuple[np.ndarray, bool]:
    """Solve A X = B by Gaussian elimination with partial pivoting (the inversion of the
    small capacitance matrix of Eqs. 9 and 14).  Returns (X, ok); ok is False when a
    pivot is zero or falls below SINGULAR_REL * ||A||_inf."""
    A = np.array(A, dtype=np.complex128)
    X = np.array(B, dtype=np.complex128)
    vec = X.ndim == 1
    if vec:
        X = X[:, None]
    p = A.shape[0]
    thresh = SINGULAR_REL * np.max(np.sum(np.abs(A), axis=1))
    for c in range(p):
        r = c + int(np.argmax(np.abs(A[c:, c])))
        if not (abs(A[r, c]) >= thresh and abs(A[r, c]) > 0.0):
            return X[:, 0] if vec else X, False
        if r != c:
            A[[c, r]] = A[[r, c]]
            X[[c, r]] = X[[r, c]]
        for rr in range(c + 1, p):
            f = A[rr, c] / A[c, c]
            A[rr, c:] -= f * A[c, c:]
            X[rr] -= f * X[c]
    for c in range(p - 1, -1, -1):
        X[c] = (X[c] - A[c, c + 1:] @ X[c + 1:]) / A[c, c]
    return (X[:, 0] if vec else X), True


def gauss_pp_batch(A: np.ndarray, B: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """The same elimination as gauss_pp over a leading batch axis: A (b,p,p), B (b,p)."""
    A = np.array(A, dtype=np.complex128)
    X = np.array(B, dtype=np.complex128)
    nb, p, _ = A.shape
    ok = np.ones(nb, dtype=bool)
    thresh = SINGULAR_REL * np.max(np.sum(np.abs(A), axis=2), axis=1)
    rows = np.arange(nb)
    for c in range(p):
        r = c + np.argmax(np.abs(A[:, c:, c]), axis=1)
        piv = A[rows, r, c]
        ok &= (np.abs(piv) >= thresh) & (np.abs(piv) > 0.0)
        Ar, Ac = A[rows, r].copy(), A[rows, c].copy()
        A[rows, c], A[rows, r] = Ar, Ac
        Xr, Xc = X[rows, r].copy(), X[rows, c].copy()
        X[rows, c], X[rows, r] = Xr, Xc
        pivot = np.where(ok, A[:, c, c], 1.0)
        for rr in range(c + 1, p):
            f = A[:, rr, c] / pivot
            A[:, rr, c:] -= f[:, None] * A[:, c, c:]
            X[:, rr] -= f * X[:, c]
    for c in range(p - 1, -1, -1):
        acc = X[:, c] - np.einsum("bk,bk->b", A[:, c, c + 1:], X[:, c + 1:])
        X[:, c] = acc / np.where(ok, A[:, c, c], 1.0)
    return X, ok


# --------------------------------------------------------------------------- dFOM
def fom(Es: Sequence[np.ndarray]) -> float:
    """Eq. 1 with F = sum over wavelengths of |E(r_m)|^2."""
    return float(sum(abs(E[-1]) ** 2 for E in Es))


def delta_fom(Gs, Es, V, dchi) -> float:
    """Exact dFOM of flipping the pixels V by dchi (Eqs. 4-9 evaluated at the monitor),
    summed over wavelengths; -inf when a capacitance matrix is singular."""
    total = 0.0
    for G, E in zip(Gs, Es):
        N = G.shape[0] - 1
        A = np.eye(len(V)) - G[np.ix_(V, V)] * dchi[None, :]
        y, ok = gauss_pp(A, E[V])
        if not ok:
            return -math.inf
        Em = E[N] + np.sum(G[N, V] * dchi * y)
        total += abs(Em) ** 2 - abs(E[N]) ** 2
    return float(total)


def evaluate_all(gs: Sequence[Geometry], spec: CandidateSpec, state, Gs, Es) -> np.ndarray:
    """dFOM for every candidate id (-inf where invalid).  Candidates with the same number
    of flipped pixels are solved together with gauss_pp_batch."""
    g = gs[0]
    nc = num_candidates(g, spec)
    out = np.full(nc, -np.inf)
    groups = {}
    for cid in range(nc):
        c = candidate(g, spec, state, cid)
        if c is not None:
            groups.setdefault(len(c[0]), []).append((cid, c[0], c[1]))
    for p, items in groups.items():
        ids = np.array([it[0] for it in items])
        V = np.stack([it[1] for it in items])
        D = np.stack([it[2] for it in items])
        tot = np.zeros(len(items))
        good = np.ones(len(items), dtype=bool)
        for G, E in zip(Gs, Es):
            N = G.shape[0] - 1
            GVV = G[V[:, :, None], V[:, None, :]]
            A = np.eye(p)[None] - GVV * D[:, None, :]
            y, ok = gauss_pp_batch(A, E[V])
            Em = E[N] + np.sum(G[N][V] * D * y, axis=1)
            tot += np.abs(Em) ** 2 - abs(E[N]) ** 2
            good &= ok
        out[ids] = np.where(good, tot, -np.inf)
    return out


# --------------------------------------------------------------------------- selection
def select_best(dfom: np.ndarray, tie_rel: float) -> Optional[int]:
    """Greedy policy: the maximum dFOM, lowest id among those within tie_rel of it;
    None when no candidate increases the FOM."""
    m = float(np.max(dfom)) if dfom.size else -math.inf
    if not m > 0.0:
        return None
    thr = m - tie_rel * abs(m)
    return int(np.flatnonzero(dfom >= thr)[0])


def select_topk(g: Geometry, spec: CandidateSpec, dfom: np.ndarray) -> List[int]:
    """Up to k improving candidates in (-dFOM, id) order, skipping any whose anchor is
    within Chebyshev distance excl_radius of an already taken one."""
    order = np.lexsort((np.arange(dfom.size), -dfom))
    taken: List[int] = []
    anchors: List[Tuple[int, int]] = []
    for c in order:
        if not dfom[c] > 0.0 or len(taken) == spec.k:
            break
        ax, ay = anchor(g, spec, int(c))
        if any(max(abs(ax - bx), abs(ay - by)) <= spec.excl_radius for bx, by in anchors):
            continue
        taken.append(int(c))
        anchors.append((ax, ay))
    return taken


EXPLORE_TOP = 4      # Sec. V: exploration draws among the top four FOM-increasing actions


def select_egreedy(dfom: np.ndarray, tie_rel: float, epsilon: float, u_explore: float,
                   u_pick: float) -> Optional[int]:
    """epsilon-greedy policy (Sec. V).  Exploit (u_explore >= epsilon): the greedy choice of
    select_best.  Explore (u_explore < epsilon): rank floor(u_pick * m) of the m <= 4 best
    improving candidates in (-dFOM, id) order (rank 0 is the best).  None when no candidate
    increases the FOM.  u_explore, u_pick are uniform numbers in [0, 1)."""
    best = select_best(dfom, tie_rel)
    if best is None:
        return None
    if not u_explore < epsilon:
        return best
    order = np.lexsort((np.arange(dfom.size), -dfom))
    top = [int(c) for c in order[:EXPLORE_TOP] if dfom[c] > 0.0]
    r = int(u_pick * len(top))
    return top[min(r, len(top) - 1)]


# --------------------------------------------------------------------------- update
def update_rows(G_rows: np.ndarray, C_rows: np.ndarray, dchi: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Eq. 10 for a block of rows r: G_new[r, :] = G_old[r, :] + G_old[r, V] D R, where
    R = G_new[V, :] from Eq. 14.  Rows are independent, which is what lets the paper
    partition G by rows (Sec. III, Fig. 2)."""
    return G_rows + C_rows @ (dchi[:, None] * R)


def apply_update(G: np.ndarray, E: np.ndarray, V, dchi) -> Tuple[np.ndarray, np.ndarray, bool]:
    """Eq. 14 then Eq. 10 for G and Eq. 4 for E, from snapshots of G's rows and columns
    at V (no symmetry shortcut).  Returns (G_new, E_new, ok)."""
    V = np.asarray(V)
    dchi = np.asarray(dchi, dtype=np.float64)
    A = np.eye(len(V)) - G[np.ix_(V, V)] * dchi[None, :]
    R, ok1 = gauss_pp(A, G[V, :])          # new rows of G at V (Eq. 14)
    y, ok2 = gauss_pp(A, E[V])             # new field at V (Eq. 9)
    if not (ok1 and ok2):
        return G, E, False
    C = G[:, V].copy()
    Gn = update_rows(G, C, dchi, R)
    En = E + C @ (dchi * y)
    return Gn, En, True


def brute_force(g: Geometry, state: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Discrete Dyson and Lippmann-Schwinger solves from the background:
    (I - G0 X) G = G0 and (I - G0 X) E = E_inc with X = diag(chi, 0)."""
    G0 = g0_matrix(g)
    x = np.zeros(g.N + 1)
    x[:g.N] = state.astype(np.float64) * contrast(g)
    M = np.eye(g.N + 1) - G0 * x[None, :]
    return np.linalg.solve(M, G0), np.linalg.solve(M, incident_field(g))


# --------------------------------------------------------------------------- drift checks
def ls_residual(g: Geometry, state: np.ndarray, E: np.ndarray) -> float:
    """Relative Lippmann-Schwinger residual of a field (discrete Eq. 3):
    ||E - E_inc - G0 X E||_2 / ||E||_2 with the dense background matrix."""
    G0 = g0_matrix(g)
    x = np.zeros(g.N + 1)
    x[:g.N] = np.asarray(state, dtype=np.float64) * contrast(g)
    r = E - incident_field(g) - G0 @ (x * E)
    return float(np.linalg.norm(r) / np.linalg.norm(E))


def exact_columns(g: Geometry, state: np.ndarray, cols) -> np.ndarray:
    """Columns of G = (I - G0 X)^{-1} G0 (discrete Eq. 2) for the given design."""
    return brute_force(g, np.asarray(state))[0][:, list(cols)]


# --------------------------------------------------------------------------- driver
class OracleProblem:
    """One design problem (one G and E per wavelength) advanced by greedy steps."""

    def __init__(self, geoms: Sequence[Geometry], spec: CandidateSpec, state=None):
        self.geoms = list(geoms)
        self.spec = spec
        g = self.geoms[0]
        self.state = (np.zeros(g.N, dtype=np.uint8) if state is None
                      else np.array(state, dtype=np.uint8))
        if state is None:
            self.Gs = [g0_matrix(gg) for gg in self.geoms]
            self.Es = [incident_field(gg) for gg in self.geoms]
        else:
            pairs = [brute_force(gg, self.state) for gg in self.geoms]
            self.Gs = [p[0] for p in pairs]
            self.Es = [p[1] for p in pairs]

    def fom(self) -> float:
        return fom(self.Es)

    def evaluate(self) -> np.ndarray:
        return evaluate_all(self.geoms, self.spec, self.state, self.Gs, self.Es)

    def choose_egreedy(self, dfom: np.ndarray, epsilon: float, u_explore: float, u_pick: float) -> List[int]:
        c = select_egreedy(dfom, self.spec.tie_rel, epsilon, u_explore, u_pick)
        return [] if c is None else [c]

    def choose(self, dfom: np.ndarray) -> List[int]:
        if self.spec.k <= 1:
            c = select_best(dfom, self.spec.tie_rel)
            return [] if c is None else [c]
        return select_topk(self.geoms[0], self.spec, dfom)

    def flip_set(self, ids: Sequence[int]) -> Tuple[np.ndarray, np.ndarray]:
        Vs, Ds = [], []
        for c in ids:
            V, d = candidate(self.geoms[0], self.spec, self.state, c)
            Vs.append(V)
            Ds.append(d)
        return np.concatenate(Vs), np.concatenate(Ds)

    def accept(self, ids: Sequence[int]) -> List[int]:
        """Apply the chosen candidates; a multi-candidate set whose joint dFOM is not
        positive falls back to its best member.  Returns the ids applied."""
        ids = list(ids)
        V, d = self.flip_set(ids)
        if len(ids) > 1 and not delta_fom(self.Gs, self.Es, V, d) > 0.0:
            ids = ids[:1]
            V, d = self.flip_set(ids)
        newG, newE = [], []
        for G, E in zip(self.Gs, self.Es):
            Gn, En, ok = apply_update(G, E, V, d)
            if not ok:
                raise FloatingPointError("singular capacitance matrix on the update path")
            newG.append(Gn)
            newE.append(En)
        self.Gs, self.Es = newG, newE
        self.state[V] ^= 1
        return ids

    def step(self) -> Tuple[List[int], np.ndarray]:
        dfom = self.evaluate()
        ids = self.choose(dfom)
        if ids:
            ids = self.accept(ids)
        return ids, dfom
