"""epsilon-greedy policy (Sec. V) on the GPU against the oracle's policy with the same
uniform numbers, run lock-step: the chosen candidate equals the oracle's unless the two are a
near tie (then the oracle's choice is applied on both sides), G and E stay within the FP64
tolerance, and every accepted action increases the FOM."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import gf_oracle as O
from paper_2202_05388_gb300 import build as BLD
from paper_2202_05388_gb300 import gfopt as B
from paper_2202_05388_gb300 import workloads as W
from paper_2202_05388_gb300.egreedy import egreedy_study, metalens_21
from paper_2202_05388_gb300.optimizer import GreedyOptimizer

from gpu_parity import GAP, TOL, compare_state, rel_err


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BLD.build()


@pytest.mark.parametrize("nx,ny,kind,ratio,beyond,eps,seed", [(12, 10, W.KIND_SINGLE, 20, 1.0, 0.3, 1),
                                                              (16, 14, W.KIND_SINGLE, 20, 1.0, 0.6, 2),
                                                              (16, 12, W.KIND_BRUSH2, 6, 2.0, 0.5, 3)])
def test_egreedy_lockstep_vs_oracle(nx, ny, kind, ratio, beyond, eps, seed):
    wl = W.small(nx, ny, kind=kind, dir_mask=3, ratio=ratio, beyond_edge=beyond)
    opt = GreedyOptimizer(wl.geoms, wl.spec)
    opt.fill()
    opt.set_egreedy(eps, seed=seed, horizon=64)
    orc = O.OracleProblem(wl.geoms, wl.spec)
    explored = 0
    steps = 0
    for t in range(25):
        opt.evaluate()
        opt.select()
        d = orc.evaluate()
        u1, u2 = opt.uniforms[t]
        want = orc.choose_egreedy(d, eps, float(u1), float(u2))
        r = opt.read_step()
        if not want:
            assert r.status == B.GF_ENOIMPROVE
            break
        assert r.status == B.GF_OK
        got = r.ids[0]
        if got != want[0]:
            # only a near tie may order differently (mirror-symmetric candidates)
            assert abs(d[got] - d[want[0]]) <= GAP * abs(d[want[0]]), (t, got, want, d[got], d[want[0]])
            opt.idx[:1].fill_(want[0])
        explored += int(u1 < eps)
        before = orc.fom()
        orc.accept(want)
        opt.update()
        torch.cuda.synchronize()
        assert orc.fom() > before
        compare_state(opt, orc, tag=f"step {t}")
        steps += 1
    assert steps >= 3 and explored >= 1


def test_egreedy_zero_epsilon_is_greedy_and_validation():
    wl = W.small(12, 10, kind=W.KIND_SINGLE, dir_mask=3)
    a = GreedyOptimizer(wl.geoms, wl.spec)
    b = GreedyOptimizer(wl.geoms, wl.spec)
    a.fill()
    b.fill()
    b.set_egreedy(0.0, seed=9)
    ra, rb = a.run(12), b.run(12)
    assert [r.ids for r in ra] == [r.ids for r in rb]
    assert torch.equal(a.G[0], b.G[0])
    u = torch.zeros(2, dtype=torch.float64, device="cuda")
    g = wl.geoms[0]
    with pytest.raises(B.GfError):
        a.h.gf_select_egreedy(g, wl.spec, a.dfom, a.ncand, 1.5, u, a.idx, a.val, a.status, a.ws, a.ws_bytes)
    k4 = W.CandidateSpec(W.KIND_SINGLE, 3, 4)
    with pytest.raises(B.GfError):
        a.h.gf_select_egreedy(g, k4, a.dfom, a.ncand, 0.1, u, a.idx, a.val, a.status, a.ws, a.ws_bytes)


def test_egreedy_study_on_the_21x21_metalens():
    """Sec. V study, reduced to 4 trajectories per epsilon: every run terminates with every
    step improving the FOM; the greedy run is deterministic."""
    res = egreedy_study(epsilons=(0.0, 0.2), trajectories=4, seed=1, max_steps=3000)
    print({e: {k: v for k, v in r.items() if k != "finals"} for e, r in res.items()})
    assert res[0.0]["trajectories"] == 1 and res[0.0]["final_fom_min"] > 1.0
    assert res[0.2]["trajectories"] == 4 and res[0.2]["final_fom_min"] > 1.0
    assert metalens_21().geoms[0].mon_y > 21 * 0.05


def test_batched_egreedy_matches_single_problem_runs():
    """The fused batch with per-problem epsilon-greedy policies (device uniform streams and step
    counters) follows exactly the trajectories of the single-problem policy, across graph replays."""
    from paper_2202_05388_gb300.batch import BatchOptimizer
    wl = W.small(12, 10, kind=W.KIND_SINGLE, dir_mask=3, ratio=20, beyond_edge=1.0)
    pols = [None, (0.3, 11), (0.6, 12), (1.0, 13)]
    bo = BatchOptimizer([wl] * len(pols), policies=pols, horizon=64)
    bo.fill()
    bo.capture(4)
    bo.replay()
    bo.replay()
    torch.cuda.synchronize()
    total = 1 + 8
    for pol, opt in zip(pols, bo.opts):
        ref = GreedyOptimizer(wl.geoms, wl.spec)
        ref.h.gf_set_update_algo(bo.update_algo)          # the fused batch's update arithmetic
        ref.fill()
        if pol is not None:
            ref.set_egreedy(pol[0], seed=pol[1], horizon=64)
        for _ in range(total):
            ref.step()
        torch.cuda.synchronize()
        assert torch.equal(opt.state, ref.state), pol
        assert float(opt.fom.cpu()[0]) == float(ref.fom.cpu()[0])
    assert int(bo._policy_steps[1].item()) == total


def test_batched_study_equals_sequential_study():
    from paper_2202_05388_gb300.egreedy import egreedy_study_batched
    a = egreedy_study(epsilons=(0.0, 0.3), trajectories=3, seed=4, max_steps=3000, update_algo=B.GF_UPDATE_TC)
    b = egreedy_study_batched(epsilons=(0.0, 0.3), trajectories=3, seed=4, max_steps=3000)
    for e in (0.0, 0.3):
        assert np.allclose(a[e]["finals"], b[e]["finals"], rtol=1e-12, atol=0), e
