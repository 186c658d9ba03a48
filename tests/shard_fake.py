"""A row-block shard held in host memory, with the step calls of a libgfopt shard written with the
oracle's own functions (candidate sets, Gaussian elimination, the selection rules and the Eq. 10
row update).  It stands in for the CUDA shard so that the driver's collectives (max of the dFOM
arrays, sum of the row panels, halo all-gather) can be run on gloo ranks without a GPU.

The shard follows the library's shard contract: it holds the rows of G of pixel rows [y0, y1)
(+ the monitor row on the last shard), the whole E and state, and reads G_VV and G[N, V] of a
candidate from its own rows and from the halo rows of pixel row y1 (G[N, V] = G[V, N] by
reciprocity).  Imported by tests only."""
import math

import numpy as np
import torch

from oracle import gf_oracle as O


class OracleShard:
    def __init__(self, geom, spec, y0, y1):
        self.g, self.spec = geom, spec
        self.y0, self.y1 = y0, y1
        nx, ny = geom.nx, geom.ny
        self.N, self.n = geom.N, geom.N + 1
        self.r0 = y0 * nx
        self.r1 = y1 * nx + (1 if y1 == ny else 0)
        self.k = max(1, spec.k)
        self.pmax = (1 if spec.kind == O.KIND_SINGLE else 4) * self.k
        self.ncand = O.num_candidates(geom, spec)
        self.dfom = torch.full((self.ncand,), -math.inf, dtype=torch.float64)
        self.idx = torch.full((self.k,), -1, dtype=torch.int32)
        self.val = torch.zeros(self.k, dtype=torch.float64)
        self.status = torch.zeros(1, dtype=torch.int32)
        self.fom = torch.zeros(1, dtype=torch.float64)
        self.applied = torch.zeros(1, dtype=torch.int32)
        self.panel = torch.zeros((self.pmax, self.n), dtype=torch.complex128)
        self.halo_rows = None

    # rows of G this shard can read: its own and, after the halo exchange, pixel row y1's
    def row(self, i):
        if self.r0 <= i < self.r1:
            return self.Gl[i - self.r0]
        h0 = self.y1 * self.g.nx
        if self.halo_rows is not None and h0 <= i < h0 + self.g.nx:
            return self.halo_rows[i - h0]
        raise KeyError(f"row {i} is neither held nor in the halo")

    def fill(self):
        G0 = O.g0_matrix(self.g)
        self.Gl = G0[self.r0:self.r1].copy()
        self.E = O.incident_field(self.g).copy()
        self.state = np.zeros(self.N, dtype=np.uint8)
        self.status.zero_()
        self.fom[0] = abs(self.E[-1]) ** 2

    def own_candidates(self):
        g, nx = self.g, self.g.nx
        if self.spec.kind == O.KIND_SINGLE:
            return list(range(self.y0 * nx, self.y1 * nx))
        P = (nx - 1) * (g.ny - 1)
        ye = min(self.y1, g.ny - 1)
        anchors = [iy * (nx - 1) + ix for iy in range(self.y0, ye) for ix in range(nx - 1)]
        return anchors + [P + a for a in anchors]

    def evaluate(self):
        d = np.full(self.ncand, -np.inf)
        Nn = self.N
        for cid in self.own_candidates():
            c = O.candidate(self.g, self.spec, self.state, cid)
            if c is None:
                continue
            V, dchi = c
            GVV = np.array([self.row(int(v))[V] for v in V])
            GNV = np.array([self.row(int(v))[Nn] for v in V])
            y, ok = O.gauss_pp(np.eye(len(V)) - GVV * dchi[None, :], self.E[V])
            if ok:
                Em = self.E[Nn] + np.sum(GNV * dchi * y)
                d[cid] = abs(Em) ** 2 - abs(self.E[Nn]) ** 2
        self.dfom[:] = torch.from_numpy(d)

    def select(self):
        d = self.dfom.numpy()
        if self.spec.k <= 1:
            c = O.select_best(d, self.spec.tie_rel)
            ids = [] if c is None else [c]
        else:
            ids = O.select_topk(self.g, self.spec, d)
        self.idx.fill_(-1)
        for q, c in enumerate(ids):
            self.idx[q] = c
            self.val[q] = float(d[c])
        self.status[0] = 0 if ids else 4

    def _update_set(self, ids):
        Vs, Ds = [], []
        for c in ids:
            V, dchi = O.candidate(self.g, self.spec, self.state, c)
            Vs.append(V)
            Ds.append(dchi)
        return np.concatenate(Vs), np.concatenate(Ds)

    def _ids(self):
        return [int(c) for c in self.idx.tolist() if c >= 0]

    def gather(self):
        self.panel.zero_()
        if int(self.status[0]) != 0:
            return
        V, _ = self._update_set(self._ids())
        for u, v in enumerate(V):
            if self.r0 <= v < self.r1:
                self.panel[u] = torch.from_numpy(self.Gl[v - self.r0])

    def apply(self):
        if int(self.status[0]) != 0:
            self.applied[0] = 0
            return
        ids = self._ids()
        V, dchi = self._update_set(ids)
        R0 = self.panel.numpy()[:len(V)]
        Nn = self.N

        def joint(Vs, ds, rows):
            y, ok = O.gauss_pp(np.eye(len(Vs)) - rows[:, Vs] * ds[None, :], self.E[Vs])
            if not ok:
                return -math.inf
            Em = self.E[Nn] + np.sum(rows[:, Nn] * ds * y)
            return abs(Em) ** 2 - abs(self.E[Nn]) ** 2

        if len(ids) > 1 and not joint(V, dchi, R0) > 0.0:      # the joint set fails: the best alone
            ids = ids[:1]
            V, dchi = self._update_set(ids)
            R0 = R0[:len(V)]
        A = np.eye(len(V)) - R0[:, V] * dchi[None, :]
        R, ok1 = O.gauss_pp(A, R0)
        y, ok2 = O.gauss_pp(A, self.E[V])
        assert ok1 and ok2
        C = self.Gl[:, V].copy()
        self.Gl = O.update_rows(self.Gl, C, dchi, R)
        self.E = self.E + R0.T @ (dchi * y)                     # G[i, V] = G[V, i]
        self.state[V] ^= 1
        self.fom[0] = abs(self.E[Nn]) ** 2
        self.applied[0] = len(ids)

    def pack_halo(self):
        nx = self.g.nx
        return torch.from_numpy(self.Gl[:nx].copy())           # the rows of pixel row y0

    def unpack_halo(self, rec):
        self.halo_rows = rec.numpy().copy()

    def step_record(self):
        return torch.cat([self.idx.to(torch.float64), self.val, self.status.to(torch.float64), self.fom,
                          self.applied.to(torch.float64)])
