"""DeferredOptimizer: one design problem in the deferred (low-rank) form -- G0 implicit, the
Eq. 10 terms stored as columns C_s and blocks M_s, the bands / monitor row / field explicit --
driven through the libgfopt gf_lowrank_* calls.  Memory O(n K) for K flipped pixels instead of
the dense form's O(n^2); every step runs in the CUDA library on the current torch stream.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np
import torch

from . import gfopt as B
from .optimizer import StepResult
from .workloads import CandidateSpec, Geometry


class DeferredOptimizer:
    def __init__(self, geom: Geometry, spec: CandidateSpec, max_cols: int, device: int = 0, handle=None):
        if not torch.cuda.is_available():
            raise B.GfError(B.GF_ECUDA, "DeferredOptimizer needs a CUDA device (no CPU fallback)")
        per = 1 if spec.kind == B.GF_KIND_SINGLE else 4
        if spec.k < 1 or spec.k * per > 32:
            raise B.GfError(B.GF_EINVAL, "the deferred form applies at most 32 pixels per step "
                                         "(k <= 32 single pixels, k <= 8 brushes)")
        self.geom = geom
        self.spec = spec
        self.device = torch.device("cuda", device)
        self.h = handle or B.Handle(device)
        N, n = geom.N, geom.N + 1
        self.N, self.n = N, n
        dev = self.device
        self.E = torch.empty(n, dtype=torch.complex128, device=dev)
        self.bands = torch.empty(B.GF_NBANDS * N, dtype=torch.complex128, device=dev)
        self.monrow = torch.empty(n, dtype=torch.complex128, device=dev)
        self.U = torch.empty((max_cols, n), dtype=torch.complex128, device=dev)     # column k = U[k]
        self.max_cols = max_cols
        self.lr = B.gf_lowrank(B.geom_struct(geom), self.E.data_ptr(), self.bands.data_ptr(), self.monrow.data_ptr(),
                               self.U.data_ptr(), int(max_cols))
        self.ws_bytes = self.h.gf_lowrank_workspace_size(geom, max_cols)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.sel_ws_bytes = self.h.gf_workspace_size(geom, 1, B.GF_C128, spec)
        self.sel_ws = torch.empty(self.sel_ws_bytes, dtype=torch.uint8, device=dev)
        self.state = torch.zeros(N, dtype=torch.uint8, device=dev)
        self.ncand = self.h.gf_num_candidates(geom, spec)
        self.dfom = torch.empty(self.ncand, dtype=torch.float64, device=dev)
        self.k = max(1, spec.k)
        self.idx = torch.full((self.k,), -1, dtype=torch.int32, device=dev)
        self.val = torch.empty(self.k, dtype=torch.float64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.fom = torch.zeros(1, dtype=torch.float64, device=dev)
        self.applied = torch.zeros(1, dtype=torch.int32, device=dev)

    def _st(self):
        return torch.cuda.current_stream(self.device)

    def init(self):
        self.h.gf_lowrank_init(self.lr, self.ws, self.ws_bytes, self._st())
        self.state.zero_()
        self.h.gf_lowrank_fom(self.lr, self.fom, self._st())

    def evaluate(self):
        self.h.gf_lowrank_eval(self.lr, self.state, self.spec, self.dfom, self._st())

    def select(self):
        self.h.gf_select_topk(self.geom, self.spec, self.dfom, self.ncand, self.idx, self.val, self.status,
                              self.sel_ws, self.sel_ws_bytes, self._st())

    def update(self):
        self.h.gf_lowrank_update(self.lr, self.state, self.spec, self.idx, self.status, self.fom, self.ws,
                                 self.ws_bytes, self._st(), applied=self.applied)

    def step(self):
        self.evaluate()
        self.select()
        self.update()

    def force(self, ids: Sequence[int]):
        self.idx.fill_(-1)
        self.idx[0] = int(ids[0])
        self.status.zero_()
        self.update()

    def read_step(self) -> StepResult:
        k = self.k
        packed = torch.cat([self.idx.to(torch.float64), self.val, self.status.to(torch.float64), self.fom]).cpu().numpy()
        ids = [int(x) for x in packed[:k] if x >= 0]
        return StepResult(ids, [float(x) for x in packed[k:k + len(ids)]], int(packed[2 * k]), float(packed[2 * k + 1]))

    def run(self, steps: int) -> List[StepResult]:
        out = []
        for _ in range(steps):
            self.step()
            r = self.read_step()
            out.append(r)
            if r.status != B.GF_OK:
                break
        return out

    def count(self):
        return self.h.gf_lowrank_count(self.lr, self.ws, self.ws_bytes, self._st())

    def materialize(self) -> torch.Tensor:
        ldg = self.n + (self.n & 1)
        G = torch.empty((self.n, ldg), dtype=torch.complex128, device=self.device)
        self.h.gf_lowrank_materialize(self.lr, G, ldg, self.ws, self.ws_bytes, self._st())
        return G[:, :self.n]
