"""Deferred (low-rank) form of the FP64 oracle, for full-size parity checks.

TEST INFRASTRUCTURE ONLY (same rules as oracle.gf_oracle).

Eq. 10 applied step after step gives G_t = G0 + sum_{s < t} C_s D_s R_s, where C_s = G_s[:, V_s],
R_s = A_s^{-1} G_s[V_s, :] (Eq. 14) and D_s = diag(d_chi of V_s).  Any entry of G_t is therefore
computable from G0's closed form plus the stored factors (n x p_s and p_s x n per step), without
materialising the n x n matrix.  The field follows Eq. 4 exactly as in the dense oracle (E is
only n long).  This class runs the same greedy steps as OracleProblem on the 192 x 192 workload
(n = 36865), where the dense G would need 21.7 GB, and exposes G entries one by one.

The arithmetic per step is that of gf_oracle: G_VV blocks and monitor rows are gathered (here:
computed entry by entry), dFOM uses gauss_pp_batch (Eqs. 4-9), selection uses select_best /
select_topk, the update solves with gauss_pp (Eq. 14).  Only the summation order of Eq. 10
differs (G0 + sum of factor products instead of sequential in-place adds), which changes
results by rounding only; tests pin it to the dense oracle on small grids.
"""
from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

from oracle import gf_oracle as O
from paper_2202_05388_gb300.workloads import CandidateSpec, Geometry, KIND_SINGLE


class LowRankProblem:
    def __init__(self, g: Geometry, spec: CandidateSpec):
        self.g = g
        self.spec = spec
        self.N = g.N
        self.n = g.N + 1
        self.pts = O.points(g)
        self.state = np.zeros(g.N, dtype=np.uint8)
        self.E = O.incident_field(g)
        self.C: List[np.ndarray] = []      # C_s (n x p_s)
        self.R: List[np.ndarray] = []      # D_s R_s (p_s x n)

    # ---- G entries
    def g0(self, i: np.ndarray, j: np.ndarray) -> np.ndarray:
        """G0[i, j] elementwise from the closed form (self term on the pixel diagonal)."""
        i = np.asarray(i)
        j = np.asarray(j)
        d = self.pts[i] - self.pts[j]
        r = np.sqrt(d[..., 0] ** 2 + d[..., 1] ** 2)
        out = np.zeros(np.broadcast(i, j).shape, dtype=np.complex128)
        off = i != j
        with np.errstate(divide="ignore", invalid="ignore"):
            out[off] = O.g0_pair(self.g, r[off])
        diag = (i == j) & (i < self.N)
        out[diag] = O.g0_self(self.g)
        return out

    def entries(self, i, j) -> np.ndarray:
        """G_t[i, j] elementwise: G0 plus every stored Eq. 10 term."""
        i = np.asarray(i)
        j = np.asarray(j)
        out = self.g0(i, j)
        for C, DR in zip(self.C, self.R):
            out = out + np.einsum("...k,k...->...", C[i], DR[:, j])
        return out

    def rows(self, V: np.ndarray) -> np.ndarray:
        """G_t[V, :] (len(V) x n)."""
        V = np.asarray(V)
        jj = np.arange(self.n)
        out = self.g0(V[:, None], jj[None, :])
        for C, DR in zip(self.C, self.R):
            out = out + C[V] @ DR
        return out

    def cols(self, V: np.ndarray) -> np.ndarray:
        """G_t[:, V] (n x len(V))."""
        V = np.asarray(V)
        ii = np.arange(self.n)
        out = self.g0(ii[:, None], V[None, :])
        for C, DR in zip(self.C, self.R):
            out = out + C @ DR[:, V]
        return out

    # ---- one greedy step
    def fom(self) -> float:
        return float(abs(self.E[-1]) ** 2)

    def evaluate(self) -> np.ndarray:
        """dFOM of every candidate with the oracle's batched elimination (Eqs. 4-9)."""
        g, spec = self.g, self.spec
        nc = O.num_candidates(g, spec)
        out = np.full(nc, -np.inf)
        groups = {}
        for cid in range(nc):
            c = O.candidate(g, spec, self.state, cid)
            if c is not None:
                groups.setdefault(len(c[0]), []).append((cid, c[0], c[1]))
        N = self.N
        for p, items in groups.items():
            ids = np.array([it[0] for it in items])
            V = np.stack([it[1] for it in items])
            D = np.stack([it[2] for it in items])
            GVV = self.entries(V[:, :, None], V[:, None, :])
            A = np.eye(p)[None] - GVV * D[:, None, :]
            y, ok = O.gauss_pp_batch(A, self.E[V])
            GNV = self.entries(np.full(V.shape, N), V)
            Em = self.E[N] + np.sum(GNV * D * y, axis=1)
            out[ids] = np.where(ok, np.abs(Em) ** 2 - abs(self.E[N]) ** 2, -np.inf)
        return out

    def choose(self, dfom: np.ndarray) -> List[int]:
        if self.spec.k <= 1:
            c = O.select_best(dfom, self.spec.tie_rel)
            return [] if c is None else [c]
        return O.select_topk(self.g, self.spec, dfom)

    def flip_set(self, ids: Sequence[int], spec: CandidateSpec = None):
        spec = spec or self.spec
        Vs, Ds = [], []
        for c in ids:
            V, d = O.candidate(self.g, spec, self.state, c)
            Vs.append(V)
            Ds.append(d)
        return np.concatenate(Vs), np.concatenate(Ds)

    def joint_dfom(self, ids: Sequence[int], spec: CandidateSpec = None) -> float:
        """dFOM of applying the candidates together (this wavelength's share); -inf if A is
        singular."""
        V, d = self.flip_set(list(ids), spec)
        GVV = self.entries(V[:, None], V[None, :])
        A = np.eye(len(V)) - GVV * d[None, :]
        y, ok = O.gauss_pp(A, self.E[V])
        if not ok:
            return -np.inf
        dE = np.sum(self.entries(np.full(len(V), self.N), V) * d * y)
        return abs(self.E[self.N] + dE) ** 2 - abs(self.E[self.N]) ** 2

    def accept(self, ids: Sequence[int], spec: CandidateSpec = None, joint_check: bool = True) -> List[int]:
        """Apply candidates; with `spec` given they are applied as that family's candidates
        (used to reach a patterned design by single-pixel toggles).  joint_check=False applies
        the set as given (the caller took the joint decision, e.g. summed over wavelengths)."""
        ids = list(ids)
        V, d = self.flip_set(ids, spec)
        if len(ids) > 1 and joint_check:
            GVV = self.entries(V[:, None], V[None, :])
            A = np.eye(len(V)) - GVV * d[None, :]
            y, ok = O.gauss_pp(A, self.E[V])
            dE = np.sum(self.entries(np.full(len(V), self.N), V) * d * y)
            joint = abs(self.E[self.N] + dE) ** 2 - abs(self.E[self.N]) ** 2
            if not (ok and joint > 0.0):
                ids = ids[:1]
                V, d = self.flip_set(ids, spec)
        Rows = self.rows(V)                      # G[V, :]
        Cols = self.cols(V)                      # G[:, V]
        A = np.eye(len(V)) - Rows[:, V] * d[None, :]
        R, ok1 = O.gauss_pp(A, Rows)             # Eq. 14
        y, ok2 = O.gauss_pp(A, self.E[V])        # Eq. 9
        if not (ok1 and ok2):
            raise FloatingPointError("singular capacitance matrix on the update path")
        self.E = self.E + Cols @ (d * y)         # Eq. 4
        self.C.append(Cols)
        self.R.append(d[:, None] * R)            # Eq. 10 term: G += C D R
        self.state[V] ^= 1
        return ids

    def step(self):
        dfom = self.evaluate()
        ids = self.choose(dfom)
        if ids:
            ids = self.accept(ids)
        return ids, dfom
