"""Batched problems through CUDA-graph replay: every problem of a small seeded batch follows
exactly the trajectory it follows when stepped alone (same flips, same G, E and FOM), and
both match the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import gf_oracle as O
from paper_2202_05388_gb300 import build as BLD
from paper_2202_05388_gb300 import gfopt as B
from paper_2202_05388_gb300 import workloads as W
from paper_2202_05388_gb300.batch import BatchOptimizer, Schedule
from paper_2202_05388_gb300.optimizer import GreedyOptimizer

from gpu_parity import rel_err


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BLD.build()


def _small_batch():
    # the batched family (single-pixel toggles, seeded sides / lambda/dx / focus), scaled down
    out = []
    rng = np.random.default_rng(5)
    for b in range(6):
        side = int(rng.choice([8, 10, 12, 14]))
        ratio = int(rng.choice([16, 20, 24]))
        out.append(W.small(side, side, kind=W.KIND_SINGLE, dir_mask=3, ratio=ratio,
                           beyond_edge=float(rng.uniform(2.0, 6.0)), steps=4))
    return out


@pytest.mark.parametrize("sch", [Schedule(1, "given"), Schedule(3, "largest_first"), Schedule(6, "given")])
def test_graph_batch_matches_single_problem_runs_and_oracle(sch):
    wls = _small_batch()
    bo = BatchOptimizer(wls)
    bo.schedule = sch
    bo.fill()
    steps = 3
    bo.capture(steps)           # one warm-up step runs during capture set-up
    bo.replay()
    torch.cuda.synchronize()
    total = steps + 1
    for wl, opt in zip(wls, bo.opts):
        ref = GreedyOptimizer(wl.geoms, wl.spec)
        ref.fill()
        orc = O.OracleProblem(wl.geoms, wl.spec)
        for _ in range(total):
            ref.step()
            orc.step()
        torch.cuda.synchronize()
        assert torch.equal(opt.state, ref.state)
        assert rel_err(opt.G[0][:, :opt.n].cpu().numpy(), ref.G[0][:, :ref.n].cpu().numpy()) <= 1e-14
        assert np.array_equal(opt.state.cpu().numpy(), orc.state)
        assert rel_err(opt.G[0][:, :opt.n].cpu().numpy(), orc.Gs[0]) <= 1e-10
        assert abs(float(opt.fom.cpu()[0]) - orc.fom()) <= 1e-10 * orc.fom()


def test_autotune_picks_a_timed_schedule():
    wls = _small_batch()
    bo = BatchOptimizer(wls)
    bo.fill()
    best = bo.autotune(candidates=[Schedule(1, "given"), Schedule(6, "largest_first")], steps=1, reps=1)
    assert best in [t[0] for t in bo.timings]
    assert min(t[1] for t in bo.timings) == [t[1] for t in bo.timings if t[0] == best][0]
