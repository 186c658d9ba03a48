"""Plain FP64 CPU oracle of the optimizer in its 3-D form (the paper's own setting).

TEST INFRASTRUCTURE ONLY (same rules as oracle.gf_oracle: only tests/, __graft_entry__.smoke()
and bench.py's CPU legs may use it; it shares no code with the CUDA path).

What it computes (Wang et al., arXiv:2202.05388, Sec. II with 3x3 dyadic blocks):
* Unknowns: the three Cartesian field components at each of the N voxels and at the monitor
  point, u = 3 * point + component; n = 3 (N + 1).
* Background dyadic Green's function of vacuum, G0(R) = (I + grad grad / k^2) e^{ikR} / (4 pi R),
  written out as e^{ikR}/(4 pi R) [A(kR) I + B(kR) R^ R^] with
  A = 1 + (i kR - 1)/(kR)^2 and B = (3 - 3 i kR - (kR)^2)/(kR)^2.  The paper's b = k^2 d_eps dV
  is folded into the matrix, G_ij = k^2 dV G0(r_i - r_j), so that a flip changes the contrast of
  every component of a voxel by d_chi = +-(eps_mat - eps_bg) (Eqs. 4-9 with b -> d_chi).
* Voxel self block: the principal-volume integral over a sphere of the voxel's volume with the
  depolarisation dyadic I/3: k^2 int G0 dV = [(2/3)((1 - i k a) e^{ika} - 1) - 1/3] I,
  a = (3 dV / (4 pi))^(1/3).  The monitor's self block is never read and set to 0.
* Incident field: x-polarised plane wave travelling +z, E_inc = x^ e^{ikz}.
* FOM = |E(r_m)|^2 summed over the three components (Eq. 1 with the focal intensity).
* Candidates: pillars -- 2x2 lateral blocks through all nz layers (Sec. IV), both directions;
  id = dir * P + iy (nx - 1) + ix with P = (nx - 1)(ny - 1), as for 2-D brushes.
* dFOM, selection and the update are those of oracle.gf_oracle applied to the 3n x 3n system
  (A = I - G_VV D over the 3 p unknowns of the flipped voxels, Eqs. 9, 10, 14, 4).
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

from oracle import gf_oracle as O
from paper_2202_05388_gb300.workloads import CandidateSpec, Geometry3D, KIND_PILLAR, DIR_FILL, DIR_CLEAR


def wavenumber(g: Geometry3D) -> float:
    return 2.0 * math.pi / g.wavelength


def points(g: Geometry3D) -> np.ndarray:
    """(N + 1, 3) voxel centres, then the monitor."""
    iz, iy, ix = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    c = np.stack([(ix.ravel() + 0.5) * g.dx, (iy.ravel() + 0.5) * g.dx, (iz.ravel() + 0.5) * g.dx], axis=1)
    return np.vstack([c, [[g.mon_x, g.mon_y, g.mon_z]]])


def dyadic(g: Geometry3D, R: np.ndarray) -> np.ndarray:
    """k^2 dV G0(R) for separation vectors R (..., 3), R != 0: (..., 3, 3) complex."""
    k = wavenumber(g)
    dV = g.dx ** 3
    r = np.linalg.norm(R, axis=-1)
    kr = k * r
    phase = np.exp(1j * kr) / (4.0 * math.pi * r)
    A = 1.0 + (1j * kr - 1.0) / kr ** 2
    Bc = (3.0 - 3.0j * kr - kr ** 2) / kr ** 2
    u = R / r[..., None]
    out = (A[..., None, None] * np.eye(3) + Bc[..., None, None] * u[..., :, None] * u[..., None, :])
    return (k * k * dV) * phase[..., None, None] * out


def self_term(g: Geometry3D) -> complex:
    """k^2 times the principal-volume integral of G0 over the equal-volume sphere, minus the
    depolarisation 1/3 (a scalar times I)."""
    k = wavenumber(g)
    a = (3.0 * g.dx ** 3 / (4.0 * math.pi)) ** (1.0 / 3.0)
    ika = 1j * k * a
    return (2.0 / 3.0) * ((1.0 - ika) * np.exp(ika) - 1.0) - 1.0 / 3.0


def g0_matrix(g: Geometry3D) -> np.ndarray:
    """The 3n x 3n background matrix (block (i, j) = k^2 dV G0(r_i - r_j))."""
    P = points(g)
    npt = g.N + 1
    R = P[:, None, :] - P[None, :, :]
    off = ~np.eye(npt, dtype=bool)
    blocks = np.zeros((npt, npt, 3, 3), dtype=np.complex128)
    blocks[off] = dyadic(g, R[off])
    s = self_term(g)
    for j in range(g.N):
        blocks[j, j] = s * np.eye(3)
    return blocks.transpose(0, 2, 1, 3).reshape(3 * npt, 3 * npt)


def incident_field(g: Geometry3D) -> np.ndarray:
    P = points(g)
    E = np.zeros((g.N + 1, 3), dtype=np.complex128)
    E[:, 0] = np.exp(1j * wavenumber(g) * P[:, 2])
    return E.ravel()


def contrast(g: Geometry3D) -> float:
    return g.eps_mat - g.eps_bg


def monitor_rows(g: Geometry3D) -> np.ndarray:
    return np.arange(3 * g.N, 3 * g.N + 3)


def fom(E: np.ndarray, g: Geometry3D) -> float:
    Em = E[monitor_rows(g)]
    return float(np.sum(np.abs(Em) ** 2))


def num_candidates(g: Geometry3D, spec: CandidateSpec) -> int:
    return 2 * (g.nx - 1) * (g.ny - 1)


def candidate(g: Geometry3D, spec: CandidateSpec, state: np.ndarray, cid: int) -> Tuple[np.ndarray, np.ndarray]:
    """Unknowns V (3 per flipped voxel, voxel-major) and their contrast changes."""
    P = (g.nx - 1) * (g.ny - 1)
    d, a = divmod(int(cid), P)
    if not (spec.dir_mask & (DIR_FILL if d == 0 else DIR_CLEAR)):
        return np.zeros(0, dtype=np.int64), np.zeros(0)
    ay, ax = divmod(a, g.nx - 1)
    if getattr(spec, "aligned", False) and (ax % 2 or ay % 2):
        return np.zeros(0, dtype=np.int64), np.zeros(0)      # Sec. IV: aligned partitions only
    target = 0 if d == 0 else 1
    vox = []
    for iz in range(g.nz):
        for dy in (0, 1):
            for dx in (0, 1):
                j = (iz * g.ny + ay + dy) * g.nx + ax + dx
                if state[j] == target:
                    vox.append(j)
    chi = contrast(g) if d == 0 else -contrast(g)
    V = np.array([3 * j + c for j in vox for c in range(3)], dtype=np.int64)
    return V, np.full(len(V), chi)


def anchor(g: Geometry3D, cid: int) -> Tuple[int, int]:
    P = (g.nx - 1) * (g.ny - 1)
    a = int(cid) % P
    ay, ax = divmod(a, g.nx - 1)
    return ax, ay


def delta_fom(g: Geometry3D, G: np.ndarray, E: np.ndarray, V, dchi) -> Optional[float]:
    """Eqs. 6-9 and Eq. 4 at the monitor: None when A is singular (partial-pivoting test)."""
    A = np.eye(len(V)) - G[np.ix_(V, V)] * np.asarray(dchi)[None, :]
    y, ok = O.gauss_pp(A, E[V][:, None])
    if not ok:
        return None
    m = monitor_rows(g)
    Em = E[m]
    dE = G[np.ix_(m, V)] @ (np.asarray(dchi) * y[:, 0])
    return float(np.sum(np.abs(Em + dE) ** 2) - np.sum(np.abs(Em) ** 2))


def evaluate_all(g: Geometry3D, spec: CandidateSpec, state, G, E) -> np.ndarray:
    out = np.full(num_candidates(g, spec), -np.inf)
    for c in range(out.size):
        V, d = candidate(g, spec, state, c)
        if V.size == 0:
            continue
        v = delta_fom(g, G, E, V, d)
        if v is not None:
            out[c] = v
    return out


def select_topk(g: Geometry3D, spec: CandidateSpec, dfom: np.ndarray) -> List[int]:
    order = np.lexsort((np.arange(dfom.size), -dfom))
    taken, anchors = [], []
    for c in order:
        if not dfom[c] > 0.0 or len(taken) == spec.k:
            break
        ax, ay = anchor(g, int(c))
        if any(max(abs(ax - bx), abs(ay - by)) <= spec.excl_radius for bx, by in anchors):
            continue
        taken.append(int(c))
        anchors.append((ax, ay))
    return taken


def brute_force(g: Geometry3D, state: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """(I - G0 X) G = G0 and (I - G0 X) E = E_inc, X = diag of the unknowns' contrasts."""
    G0 = g0_matrix(g)
    x = np.zeros(3 * (g.N + 1))
    x[:3 * g.N] = np.repeat(np.asarray(state, dtype=np.float64), 3) * contrast(g)
    M = np.eye(x.size) - G0 * x[None, :]
    return np.linalg.solve(M, G0), np.linalg.solve(M, incident_field(g))


class OracleProblem3D:
    def __init__(self, g: Geometry3D, spec: CandidateSpec):
        self.g = g
        self.spec = spec
        self.state = np.zeros(g.N, dtype=np.uint8)
        self.G = g0_matrix(g)
        self.E = incident_field(g)

    def fom(self) -> float:
        return fom(self.E, self.g)

    def evaluate(self) -> np.ndarray:
        return evaluate_all(self.g, self.spec, self.state, self.G, self.E)

    def choose(self, dfom: np.ndarray) -> List[int]:
        if self.spec.k <= 1:
            c = O.select_best(dfom, self.spec.tie_rel)
            return [] if c is None else [c]
        return select_topk(self.g, self.spec, dfom)

    def flip_set(self, ids: Sequence[int]):
        Vs, Ds = [], []
        for c in ids:
            V, d = candidate(self.g, self.spec, self.state, c)
            Vs.append(V)
            Ds.append(d)
        return np.concatenate(Vs), np.concatenate(Ds)

    def accept(self, ids: Sequence[int]) -> List[int]:
        ids = list(ids)
        V, d = self.flip_set(ids)
        if len(ids) > 1 and not (delta_fom(self.g, self.G, self.E, V, d) or -1.0) > 0.0:
            ids = ids[:1]
            V, d = self.flip_set(ids)
        Gn, En, ok = O.apply_update(self.G, self.E, V, d)
        if not ok:
            raise FloatingPointError("singular capacitance matrix on the update path")
        self.G, self.E = Gn, En
        self.state[np.unique(V // 3)] ^= 1
        return ids

    def step(self):
        dfom = self.evaluate()
        ids = self.choose(dfom)
        if ids:
            ids = self.accept(ids)
        return ids, dfom
