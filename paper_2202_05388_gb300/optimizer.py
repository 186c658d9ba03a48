"""GreedyOptimizer: the public Python entry point that owns one design problem's device
state (G, E and the bands per wavelength, the design state and the step buffers, all torch
CUDA tensors) and drives the libgfopt C ABI for each greedy step (Fig. 1 of the paper:
evaluate every candidate, select, update).  Everything runs asynchronously on the current
torch stream; only ``read_step``/``run`` copy the small step result back to the host.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import gfopt as B
from .workloads import CandidateSpec, Geometry


@dataclass
class StepResult:
    ids: List[int]          # candidate ids selected (before the joint-dFOM fallback)
    dfom: List[float]       # their individual dFOM
    status: int             # GF_OK, GF_ENOIMPROVE or GF_ESINGULAR
    fom: float              # FOM after the step


class GreedyOptimizer:
    def __init__(self, geoms: Sequence[Geometry], spec: CandidateSpec, dtype: str = "c128",
                 device: int = 0, handle: Optional[B.Handle] = None):
        if not torch.cuda.is_available():
            raise B.GfError(B.GF_ECUDA, "GreedyOptimizer needs a CUDA device (no CPU fallback)")
        self.geoms = list(geoms)
        self.spec = spec
        self.dtype = B.GF_C128 if dtype == "c128" else B.GF_C64
        self.device = torch.device("cuda", device)
        self.h = handle or B.Handle(device)
        g = self.geoms[0]
        N, n = g.N, g.N + 1
        self.N, self.n = N, n
        self.ldg = n + (n & 1)
        tdt = torch.complex128 if self.dtype == B.GF_C128 else torch.complex64
        dev = self.device
        nlam = len(self.geoms)
        self.G = [torch.empty((n, self.ldg), dtype=tdt, device=dev) for _ in range(nlam)]
        self.E = [torch.empty(n, dtype=torch.complex128, device=dev) for _ in range(nlam)]
        self.bands = [torch.empty(B.GF_NBANDS * N, dtype=torch.complex128, device=dev)
                      for _ in range(nlam)]
        self.state = torch.zeros(N, dtype=torch.uint8, device=dev)
        self.ncand = self.h.gf_num_candidates(g, spec)
        self.dfom = torch.empty(self.ncand, dtype=torch.float64, device=dev)
        k = max(1, spec.k)
        self.idx = torch.full((k,), -1, dtype=torch.int32, device=dev)
        self.val = torch.empty(k, dtype=torch.float64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.fom = torch.zeros(1, dtype=torch.float64, device=dev)
        self.applied = torch.zeros(1, dtype=torch.int32, device=dev)
        self.ws_bytes = self.h.gf_workspace_size(g, nlam, self.dtype, spec)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.probs = [B.problem_struct(gg, self.G[l], self.ldg, self.E[l], self.bands[l])
                      for l, gg in enumerate(self.geoms)]
        self.epsilon = None          # None: greedy policy; else the epsilon-greedy policy

    def set_egreedy(self, epsilon: float, seed: int, horizon: int = 4096):
        """epsilon-greedy policy (Sec. V).  The two uniform numbers of every step are drawn
        up front on the host (numpy PCG64, seeded) and kept on the device; step t reads row
        t (``uniforms`` holds them for replays and checks)."""
        self.epsilon = float(epsilon)
        self.uniforms = np.random.default_rng(seed).random((horizon, 2))
        self._u = torch.tensor(self.uniforms, dtype=torch.float64, device=self.device)
        self._t = 0

    # ---- stages (asynchronous on the current stream)
    def _st(self):
        return torch.cuda.current_stream(self.device)

    def fill(self):
        for p in self.probs:
            self.h.gf_fill_g0(p, self.dtype, self.ws, self.ws_bytes, self._st())
        self.state.zero_()
        self.h.gf_fom(self.probs, self.dtype, self.fom, self._st())

    def evaluate(self):
        self.h.gf_eval_candidates(self.probs, self.dtype, self.state, self.spec, self.dfom, self._st())

    def select(self):
        if self.epsilon is not None:
            if self._t >= self._u.shape[0]:
                raise IndexError("epsilon-greedy horizon exhausted; call set_egreedy with a larger horizon")
            self.h.gf_select_egreedy(self.geoms[0], self.spec, self.dfom, self.ncand, self.epsilon,
                                     self._u[self._t], self.idx, self.val, self.status, self.ws, self.ws_bytes,
                                     self._st())
            self._t += 1
            return
        self.h.gf_select_topk(self.geoms[0], self.spec, self.dfom, self.ncand, self.idx, self.val,
                              self.status, self.ws, self.ws_bytes, self._st())

    def update(self):
        self.h.gf_apply_update(self.probs, self.dtype, self.state, self.spec, self.idx, self.status,
                               self.fom, self.ws, self.ws_bytes, self._st(), applied=self.applied)

    def step(self):
        self.evaluate()
        self.select()
        self.update()

    def force(self, ids: Sequence[int], spec: Optional[CandidateSpec] = None):
        """Apply the given candidate ids regardless of their dFOM (tests, replays)."""
        spec = spec or self.spec
        k = max(1, spec.k)
        idx = torch.full((k,), -1, dtype=torch.int32)
        idx[:len(ids)] = torch.tensor(list(ids), dtype=torch.int32)
        if self.idx.numel() < k:
            self.idx = torch.full((k,), -1, dtype=torch.int32, device=self.device)
        self.idx[:k].copy_(idx.to(self.device))
        self.status.zero_()
        self.h.gf_apply_update(self.probs, self.dtype, self.state, spec, self.idx, self.status,
                               self.fom, self.ws, self.ws_bytes, self._st(), applied=self.applied)

    def _refresh_ws(self, restart: int):
        need = self.h.gf_refresh_workspace_size(self.geoms[0], restart)
        if getattr(self, "_rws", None) is None or self._rws.numel() < need:
            self._rws = torch.empty(need, dtype=torch.uint8, device=self.device)
        return self._rws

    def refresh(self, cols: Optional[Sequence[int]] = None, nsample: int = 8, restart: int = 30,
                max_iter: int = 300, tol: Optional[float] = None, seed: int = 0):
        """Drift check of every wavelength: Lippmann-Schwinger residual of E and GMRES re-solves
        of sampled columns of G (blocking).  Returns a list (per wavelength) of
        (residuals, iterations, column residuals)."""
        if tol is None:                      # well below the storage precision of G
            tol = 1e-12 if self.dtype == B.GF_C128 else 1e-8
        if cols is None:
            rng = np.random.default_rng(seed)
            cols = sorted(set(int(c) for c in rng.integers(0, self.n, nsample)))
        ws = self._refresh_ws(restart)
        return [self.h.gf_refresh(p, self.dtype, self.state, list(cols), restart, max_iter, tol, ws, ws.numel(),
                                  self._st()) for p in self.probs]

    # Field repair tolerances: the Eq. 3 residual a field may carry before it is re-solved (well
    # above the rounding the FP64 field accumulates from the stored G: ~1e-15 per step for
    # complex128, ~1e-7 per step for complex64 storage), and the GMRES target of the re-solve.
    E_TOL = {B.GF_C128: 1e-9, B.GF_C64: 1e-5}
    E_GMRES_TOL = 1e-13

    def refresh_fields(self, e_tol: Optional[float] = None, restart: int = 30, max_iter: int = 600):
        """Eq. 3 check of every wavelength's field; a field whose residual exceeds e_tol is
        replaced by its GMRES solution (gf_refresh_field), and the FOM is rewritten from the
        fields (gf_fom).  Blocking.  Returns one report per wavelength."""
        e_tol = self.E_TOL[self.dtype] if e_tol is None else e_tol
        ws = self._refresh_ws(restart)
        reps = [self.h.gf_refresh_field(p, self.dtype, self.state, e_tol, restart, max_iter, self.E_GMRES_TOL, ws,
                                        ws.numel(), self._st()) for p in self.probs]
        if any(r["e_replaced"] for r in reps):
            self.h.gf_fom(self.probs, self.dtype, self.fom, self._st())
        return reps

    # ---- host readback
    def read_step(self) -> StepResult:
        k = max(1, self.spec.k)
        packed = torch.cat([self.idx[:k].to(torch.float64), self.val[:k],
                            self.status.to(torch.float64), self.fom]).cpu().numpy()
        ids = [int(x) for x in packed[:k] if x >= 0]
        return StepResult(ids, [float(x) for x in packed[k:k + len(ids)]], int(packed[2 * k]),
                          float(packed[2 * k + 1]))

    def run(self, steps: int, refresh_every: int = 0, e_tol: Optional[float] = None) -> List[StepResult]:
        """Up to `steps` greedy steps, stopping at the first non-OK status.  With refresh_every
        = R > 0, every R accepted steps the fields are checked and repaired (refresh_fields);
        the reports go to self.refresh_log as (step, reports, seconds)."""
        out = []
        self.refresh_log = []
        for t in range(steps):
            self.step()
            r = self.read_step()
            out.append(r)
            if r.status != B.GF_OK:
                break
            if refresh_every and (t + 1) % refresh_every == 0:
                import time
                t0 = time.perf_counter()
                reps = self.refresh_fields(e_tol)
                self.refresh_log.append((t + 1, reps, time.perf_counter() - t0))
                if any(rep["e_replaced"] for rep in reps):
                    out[-1] = StepResult(r.ids, r.dfom, r.status, float(self.fom.cpu()[0]))
        return out

    def state_host(self) -> np.ndarray:
        return self.state.cpu().numpy()


class GreedyOptimizer3D:
    """One 3-D problem (dyadic G over the 3 (N + 1) unknowns, pillar candidates) driven
    through the gf3_* calls; the same stages and read-back as GreedyOptimizer."""

    def __init__(self, geom, spec: CandidateSpec, dtype: str = "c64", device: int = 0,
                 handle: Optional[B.Handle] = None):
        if not torch.cuda.is_available():
            raise B.GfError(B.GF_ECUDA, "GreedyOptimizer3D needs a CUDA device (no CPU fallback)")
        self.geom = geom
        self.spec = spec
        self.dtype = B.GF_C128 if dtype == "c128" else B.GF_C64
        self.device = torch.device("cuda", device)
        self.h = handle or B.Handle(device)
        self.N = geom.nx * geom.ny * geom.nz
        self.n = self.h.gf3_num_unknowns(geom)
        self.ldg = self.n + (self.n & 1)
        tdt = torch.complex128 if self.dtype == B.GF_C128 else torch.complex64
        dev = self.device
        self.G = torch.empty((self.n, self.ldg), dtype=tdt, device=dev)
        self.E = torch.empty(self.n, dtype=torch.complex128, device=dev)
        self.state = torch.zeros(self.N, dtype=torch.uint8, device=dev)
        self.ncand = self.h.gf3_num_candidates(geom)
        self.dfom = torch.empty(self.ncand, dtype=torch.float64, device=dev)
        k = max(1, spec.k)
        self.idx = torch.full((k,), -1, dtype=torch.int32, device=dev)
        self.val = torch.empty(k, dtype=torch.float64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.fom = torch.zeros(1, dtype=torch.float64, device=dev)
        self.applied = torch.zeros(1, dtype=torch.int32, device=dev)
        self.ws_bytes = self.h.gf3_workspace_size(geom, self.dtype, spec)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.prob = B.problem3d_struct(geom, self.G, self.ldg, self.E)

    def _st(self):
        return torch.cuda.current_stream(self.device)

    def fill(self):
        self.h.gf3_fill_g0(self.prob, self.dtype, self.ws, self.ws_bytes, self._st())
        self.state.zero_()
        self.h.gf3_fom(self.prob, self.dtype, self.fom, self._st())

    def evaluate(self):
        self.h.gf3_eval_candidates(self.prob, self.dtype, self.state, self.spec, self.dfom, self._st())

    def select(self):
        self.h.gf3_select_topk(self.geom, self.spec, self.dfom, self.ncand, self.idx, self.val, self.status, self.ws,
                               self.ws_bytes, self._st())

    def update(self):
        self.h.gf3_apply_update(self.prob, self.dtype, self.state, self.spec, self.idx, self.status, self.fom,
                                self.ws, self.ws_bytes, self._st(), applied=self.applied)

    def step(self):
        self.evaluate()
        self.select()
        self.update()

    def read_step(self) -> StepResult:
        k = max(1, self.spec.k)
        packed = torch.cat([self.idx[:k].to(torch.float64), self.val[:k],
                            self.status.to(torch.float64), self.fom]).cpu().numpy()
        ids = [int(x) for x in packed[:k] if x >= 0]
        return StepResult(ids, [float(x) for x in packed[k:k + len(ids)]], int(packed[2 * k]), float(packed[2 * k + 1]))
