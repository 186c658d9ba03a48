"""The deferred (G0 + stored Eq. 10 terms) oracle reproduces the dense FP64 oracle step by
step on small grids, so it can stand in for it at sizes where G does not fit in host RAM."""
import numpy as np
import pytest

from oracle import gf_oracle as O
from oracle.lowrank import LowRankProblem
from paper_2202_05388_gb300 import workloads as W


@pytest.mark.parametrize("kind,k,seed,steps", [(W.KIND_SINGLE, 1, None, 6), (W.KIND_BRUSH2, 1, 41, 5),
                                               (W.KIND_BRUSH2, 3, 42, 3)])
def test_lowrank_oracle_matches_dense_oracle(kind, k, seed, steps):
    wl = W.small(14, 11, kind=kind, dir_mask=3, k=k, excl_radius=3)
    g = wl.geoms[0]
    dense = O.OracleProblem(wl.geoms, wl.spec)
    lazy = LowRankProblem(g, wl.spec)
    if seed is not None:
        single = W.CandidateSpec(W.KIND_SINGLE, 3, 1)
        for j in np.flatnonzero(W.random_state(g.N, seed=seed, fill=0.3)):
            V, d = O.candidate(g, single, dense.state, int(j))
            dense.Gs[0], dense.Es[0], _ = O.apply_update(dense.Gs[0], dense.Es[0], V, d)
            dense.state[V] ^= 1
            lazy.accept([int(j)], single)
    taken = 0
    for _ in range(steps):
        ids_d, d_d = dense.step()
        ids_l, d_l = lazy.step()
        fin = np.isfinite(d_d)
        assert np.array_equal(fin, np.isfinite(d_l))
        assert np.max(np.abs(d_d[fin] - d_l[fin])) <= 1e-12 * max(1.0, np.max(np.abs(d_d[fin])))
        assert ids_d == ids_l
        if not ids_d:
            break
        taken += 1
        assert np.max(np.abs(dense.Es[0] - lazy.E)) <= 1e-12
        rng = np.random.default_rng(taken)
        i = rng.integers(0, g.n, 200)
        j = rng.integers(0, g.n, 200)
        assert np.max(np.abs(dense.Gs[0][i, j] - lazy.entries(i, j))) <= 1e-13
        assert np.max(np.abs(dense.Gs[0] - lazy.rows(np.arange(g.n)))) <= 1e-13
    assert taken >= 1
