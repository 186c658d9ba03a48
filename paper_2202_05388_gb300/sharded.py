"""Row-sharded optimizer: one problem's G split by rows over the ranks of a process group, the
partitioned form of the paper's method (Sec. III: partition-local dFOM, CombineGlobally, the
chosen pixels' rows broadcast to every partition, each partition updating its own rows).

Each rank holds the rows of G of a band of pixel rows (split_rows) and drives the gf_shard_* calls
of libgfopt on its GPU.  The exchanges of a step are three collectives on the process group:
  * elementwise MAX of the dFOM arrays (every rank wrote -inf outside its own candidates), so that
    every rank holds the whole array and gf_select_topk makes the same choice everywhere (the
    exact top-k merge, tie rule and exclusion zones included);
  * SUM of the row panels (each row of the update set is nonzero on its owner only): the owner
    broadcast of G[V, :];
  * all-gather of the halo records (bands and monitor entries of each shard's first pixel row,
    which the previous shard's candidates read).
With NCCL the collectives run on the device buffers; with gloo they are staged through host memory.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import torch

from . import gfopt as B
from .optimizer import StepResult
from .workloads import CandidateSpec, Geometry


def split_rows(ny: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous bands of pixel rows, as even as possible (the first ny % world bands one row
    longer), one per rank; every band holds at least one row."""
    if world < 1 or world > ny:
        raise ValueError(f"cannot split {ny} pixel rows over {world} shards")
    base, extra = divmod(ny, world)
    out, y = [], 0
    for r in range(world):
        h = base + (1 if r < extra else 0)
        out.append((y, y + h))
        y += h
    return out


class Comm:
    """Collectives over a torch.distributed process group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.host = dist.get_backend(group) == "gloo"

    def _run(self, t: torch.Tensor, fn):
        if self.host and t.is_cuda:
            h = t.cpu()
            fn(h)
            t.copy_(h)
        else:
            fn(t)

    @staticmethod
    def _real(t: torch.Tensor) -> torch.Tensor:
        return torch.view_as_real(t) if t.is_complex() else t

    def max_(self, t: torch.Tensor):
        self._run(t, lambda x: self.dist.all_reduce(x, op=self.dist.ReduceOp.MAX, group=self.group))

    def sum_(self, t: torch.Tensor):
        self._run(t, lambda x: self.dist.all_reduce(self._real(x), op=self.dist.ReduceOp.SUM, group=self.group))

    def allgather(self, t: torch.Tensor) -> List[torch.Tensor]:
        src = t.cpu() if (self.host and t.is_cuda) else t
        outs = [torch.empty_like(src) for _ in range(self.world)]
        self.dist.all_gather([self._real(o) for o in outs], self._real(src), group=self.group)
        return [o.to(t.device) for o in outs]


class LibShard:
    """One shard's device state (its rows of G; whole E and state; bands and monitor entries of
    its rows and the halo row) and the libgfopt calls of a step."""

    def __init__(self, geom: Geometry, spec: CandidateSpec, dtype: str, y0: int, y1: int, device: int = 0,
                 handle: Optional[B.Handle] = None):
        if not torch.cuda.is_available():
            raise B.GfError(B.GF_ECUDA, "LibShard needs a CUDA device (no CPU fallback)")
        self.geom, self.spec = geom, spec
        self.dtype = B.GF_C128 if dtype == "c128" else B.GF_C64
        self.device = torch.device("cuda", device)
        self.h = handle or B.Handle(device)
        N, n = geom.N, geom.N + 1
        self.N, self.n = N, n
        self.ldg = n + (n & 1)
        self.y0, self.y1 = y0, y1
        tdt = torch.complex128 if self.dtype == B.GF_C128 else torch.complex64
        dev = self.device
        self.rows = (y1 - y0) * geom.nx + (1 if y1 == geom.ny else 0)
        self.G = torch.empty((self.rows, self.ldg), dtype=tdt, device=dev)
        self.E = torch.empty(n, dtype=torch.complex128, device=dev)
        self.bands = torch.zeros(B.GF_NBANDS * N, dtype=torch.complex128, device=dev)
        self.mon = torch.zeros(n, dtype=torch.complex128, device=dev)
        self.state = torch.zeros(N, dtype=torch.uint8, device=dev)
        self.ncand = self.h.gf_num_candidates(geom, spec)
        self.dfom = torch.empty(self.ncand, dtype=torch.float64, device=dev)
        k = max(1, spec.k)
        self.k = k
        self.idx = torch.full((k,), -1, dtype=torch.int32, device=dev)
        self.val = torch.empty(k, dtype=torch.float64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.fom = torch.zeros(1, dtype=torch.float64, device=dev)
        self.applied = torch.zeros(1, dtype=torch.int32, device=dev)
        self.pmax = (1 if spec.kind == B.GF_KIND_SINGLE else 4) * k
        self.panel = torch.zeros((self.pmax, self.ldg), dtype=tdt, device=dev)
        self.halo = torch.empty((B.GF_NBANDS + 1) * geom.nx, dtype=torch.complex128, device=dev)
        self.ws_bytes = self.h.gf_workspace_size(geom, 1, self.dtype, spec)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.sh = B.gf_shard(B.geom_struct(geom), int(y0), int(y1), self.G.data_ptr(), int(self.ldg),
                             self.E.data_ptr(), self.bands.data_ptr(), self.mon.data_ptr())
        if self.h.gf_shard_rows(self.sh) != self.rows:
            raise B.GfError(B.GF_EINVAL, "shard rows disagree with the library")

    def _st(self):
        return torch.cuda.current_stream(self.device)

    def fill(self):
        self.h.gf_shard_fill_g0(self.sh, self.dtype, self.ws, self.ws_bytes, self._st())
        self.state.zero_()
        self.status.zero_()
        prob = B.problem_struct(self.geom, self.G, self.ldg, self.E, self.bands)
        self.h.gf_fom([prob], self.dtype, self.fom, self._st())

    def evaluate(self):
        self.h.gf_shard_eval(self.sh, self.dtype, self.state, self.spec, self.dfom, self._st())

    def select(self):
        self.h.gf_select_topk(self.geom, self.spec, self.dfom, self.ncand, self.idx, self.val, self.status, self.ws,
                              self.ws_bytes, self._st())

    def gather(self, spec: Optional[CandidateSpec] = None):
        """spec: another candidate family than the shard's (forced flips); its k must not exceed
        the shard's panel rows."""
        self.h.gf_shard_gather_rows(self.sh, self.dtype, self.state, spec or self.spec, self.idx, self.status,
                                    self.panel, self.ldg, self._st())

    def apply(self, spec: Optional[CandidateSpec] = None):
        self.h.gf_shard_apply_update(self.sh, self.dtype, self.state, spec or self.spec, self.idx, self.panel,
                                     self.ldg, self.status, self.fom, self.ws, self.ws_bytes, self._st(),
                                     applied=self.applied)

    def pack_halo(self) -> torch.Tensor:
        self.h.gf_shard_pack_halo(self.sh, self.halo, self._st())
        return self.halo

    def unpack_halo(self, rec: torch.Tensor):
        self.h.gf_shard_unpack_halo(self.sh, rec, self._st())

    def step_record(self) -> torch.Tensor:
        return torch.cat([self.idx.to(torch.float64), self.val, self.status.to(torch.float64), self.fom,
                          self.applied.to(torch.float64)])


class ShardedOptimizer:
    """The greedy step of one problem over the ranks of `comm` (each rank: one LibShard, or any
    object with the same methods and buffers)."""

    def __init__(self, geom: Geometry, spec: CandidateSpec, dtype: str = "c128", comm: Optional[Comm] = None,
                 device: int = 0, shard=None):
        self.comm = comm or Comm()
        self.geom, self.spec = geom, spec
        self.bands_of_rank = split_rows(geom.ny, self.comm.world)
        y0, y1 = self.bands_of_rank[self.comm.rank]
        self.shard = shard or LibShard(geom, spec, dtype, y0, y1, device)

    def _halo(self):
        recs = self.comm.allgather(self.shard.pack_halo())
        if self.comm.rank + 1 < self.comm.world:
            self.shard.unpack_halo(recs[self.comm.rank + 1])

    def fill(self):
        self.shard.fill()
        self._halo()

    def step(self):
        s = self.shard
        s.evaluate()                 # partition-local dFOM, -inf elsewhere
        self.comm.max_(s.dfom)       # CombineGlobally: every rank holds the whole array
        s.select()                   # the same choice on every rank
        s.gather()                   # this rank's rows of the update set
        self.comm.sum_(s.panel)      # the owners' broadcast of G[V, :]
        s.apply()                    # capacitance solve, own rows of G, whole E, own bands
        self._halo()

    def read_step(self) -> StepResult:
        k = self.shard.k
        packed = self.shard.step_record().cpu().numpy()
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
