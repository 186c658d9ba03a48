"""Batched problems through CUDA-graph replay, with the fused schedules (the library's batch
entry points: the persistent step kernel with several launch shapes, or one launch per stage)
and the stream-branch schedules: every problem of a small seeded batch follows exactly the
trajectory it follows when stepped alone (same flips, same G, E and FOM), and the complex128
runs match the FP64 oracle."""
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


def _small_batch(count=6, sides=(8, 10, 12, 14), kind=W.KIND_SINGLE, ratios=(16, 20, 24), dtype="c128",
                 seed=5):
    # the batched family (seeded sides / lambda/dx / focus), scaled down
    out = []
    rng = np.random.default_rng(seed)
    for b in range(count):
        side = int(rng.choice(list(sides)))
        ratio = int(rng.choice(list(ratios)))
        out.append(W.small(side, side, kind=kind, dir_mask=3, ratio=ratio,
                           beyond_edge=float(rng.uniform(2.0, 6.0)), steps=4, dtype=dtype))
    return out


def _pattern(opt, seed):
    """Seeded patterned start (forced single-pixel toggles)."""
    single = W.CandidateSpec(W.KIND_SINGLE, 3, 1)
    for j in np.flatnonzero(W.random_state(opt.N, seed=seed, fill=0.3)):
        opt.force([int(j)], single)


def _check_against_single_runs(wls, bo, total, dtype, oracle, patterned=False, start=None):
    """Each problem of the batch against its own single-problem run with the batch's update
    arithmetic (the same on every schedule: the FP64 FMA form for these small complex128
    problems by default, or the tensor-core forms)."""
    improved = 0
    for b, (wl, opt) in enumerate(zip(wls, bo.opts)):
        ref = GreedyOptimizer(wl.geoms, wl.spec, dtype=dtype)
        ref.h.gf_set_update_algo(bo.update_algo)
        ref.fill()
        if patterned:
            _pattern(ref, 100 + b)
        orc = O.OracleProblem(wl.geoms, wl.spec) if oracle else None
        for _ in range(total):
            ref.step()
            if orc is not None:
                orc.step()
        torch.cuda.synchronize()
        assert torch.equal(opt.state, ref.state)
        assert int(opt.status.cpu()[0]) == int(ref.status.cpu()[0])
        assert rel_err(opt.G[0][:, :opt.n].cpu().numpy(), ref.G[0][:, :ref.n].cpu().numpy()) <= 1e-14
        assert rel_err(opt.E[0].cpu().numpy(), ref.E[0].cpu().numpy()) <= 1e-14
        assert rel_err(opt.bands[0].cpu().numpy(), ref.bands[0].cpu().numpy()) <= 1e-14
        assert float(opt.fom.cpu()[0]) == float(ref.fom.cpu()[0])
        improved += int(not torch.equal(ref.state, start[b])) if patterned else int(ref.state.sum().item() > 0)
        if orc is not None:
            assert np.array_equal(opt.state.cpu().numpy(), orc.state)
            assert rel_err(opt.G[0][:, :opt.n].cpu().numpy(), orc.Gs[0]) <= 1e-10
            assert abs(float(opt.fom.cpu()[0]) - orc.fom()) <= 1e-10 * orc.fom()
    assert improved > 0, "no problem of the batch accepted a flip"


PERSIST, STAGED = B.GF_BATCH_PERSISTENT, B.GF_BATCH_STAGED


@pytest.mark.parametrize("sch", [Schedule(0, "given", True), Schedule(0, "given", True, 0, PERSIST, 0, 2),
                                 Schedule(3, "given", True),
                                 Schedule(0, "given", True, 0, STAGED), Schedule(3, "given", True, 0, STAGED),
                                 # one CTA takes every item in queue order (no wait can block), a few
                                 # CTAs wait on one another, work items of 4 and 16 units per thread
                                 Schedule(0, "given", True, 0, PERSIST, 1), Schedule(0, "given", True, 0, PERSIST, 3),
                                 Schedule(0, "given", True, 0, PERSIST, 0, 4), Schedule(0, "given", True, 0, PERSIST, 7, 16),
                                 Schedule(1, "given"), Schedule(3, "largest_first"), Schedule(6, "given")])
def test_graph_batch_matches_single_problem_runs_and_oracle(sch):
    wls = _small_batch()
    bo = BatchOptimizer(wls)
    assert bo.c128_fma                          # small problems: the FP64 FMA update in the batch
    bo.schedule = sch
    bo.fill()
    steps = 3
    bo.capture(steps)           # one warm-up step runs during capture set-up
    bo.replay()
    torch.cuda.synchronize()
    _check_against_single_runs(wls, bo, steps + 1, "c128", oracle=True)


@pytest.mark.parametrize("dtype,kind,count,form", [
    ("c64", W.KIND_SINGLE, 6, (PERSIST, 0, 1, 32)), ("c64", W.KIND_SINGLE, 6, (PERSIST, 2, 1, 16)),
    ("c64", W.KIND_SINGLE, 6, (PERSIST, 0, 2, 64)), ("c64", W.KIND_SINGLE, 6, (PERSIST, 0, 1, 0)),
    ("c64", W.KIND_SINGLE, 6, (STAGED, 0, 1, 32)),
    ("c128", W.KIND_BRUSH2, 5, (PERSIST, 0, 1, 32)), ("c128", W.KIND_BRUSH2, 5, (STAGED, 0, 1, 32)),
    ("c64", W.KIND_BRUSH2, 5, (PERSIST, 0, 1, 32)), ("c64", W.KIND_BRUSH2, 5, (PERSIST, 1, 1, 16)),
    ("c128", W.KIND_SINGLE, 70, (PERSIST, 0, 1, 32)), ("c128", W.KIND_SINGLE, 70, (STAGED, 0, 1, 32))])
def test_fused_batch_kinds_dtypes_and_groups(dtype, kind, count, form):
    """Complex64 items (FP32 update in 16-, 32- and 64-row tiles), brush candidates and more
    items than one launch takes (two groups), in the persistent and the staged form, behave
    exactly like the single-problem calls."""
    if kind == W.KIND_BRUSH2:
        wls = _small_batch(count, sides=(10, 12, 14), kind=kind, ratios=(20,), dtype=dtype, seed=7)
    elif count > B.BATCH_MAX:
        wls = _small_batch(count, sides=(4, 5, 6), dtype=dtype, seed=8)
    else:
        wls = _small_batch(count, dtype=dtype)
    bo = BatchOptimizer(wls, dtype=dtype)
    assert bo.schedule.fused
    bo.schedule = Schedule(0, "given", True, 0, form[0], form[1], form[2], form[3])
    bo.fill()
    patterned = kind == W.KIND_BRUSH2        # brushes rarely improve a vacuum start
    if patterned:
        for b, opt in enumerate(bo.opts):
            _pattern(opt, 100 + b)
    start = [o.state.clone() for o in bo.opts]
    bo.capture(2)
    bo.replay()
    torch.cuda.synchronize()
    _check_against_single_runs(wls, bo, 3, dtype, oracle=False, patterned=patterned, start=start)
    assert bo.total_applied() > 0


def test_autotune_picks_a_timed_schedule():
    wls = _small_batch()
    bo = BatchOptimizer(wls)
    bo.fill()
    best = bo.autotune(candidates=[Schedule(1, "given"), Schedule(6, "largest_first")], steps=1, reps=1)
    assert best in [t[0] for t in bo.timings]
    assert min(t[1] for t in bo.timings) == [t[1] for t in bo.timings if t[0] == best][0]


def test_batch_create_validates_every_item():
    wls = _small_batch(3)
    bo = BatchOptimizer(wls)
    h = bo.h
    o = bo.opts[0]
    item = B.gf_batch_item(o.probs[0], o.state.data_ptr(), o.dfom.data_ptr(), o.idx.data_ptr(), o.val.data_ptr(),
                           o.status.data_ptr(), o.fom.data_ptr(), 0, o.ws.data_ptr(), o.ws_bytes)
    tb = h.gf_batch_table_size(1)
    table = torch.empty(tb, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.GfError, match="k = 1"):
        h.gf_batch_create([item], o.dtype, W.CandidateSpec(W.KIND_SINGLE, 3, 2), table, tb)
    with pytest.raises(B.GfError) as e:
        h.gf_batch_create([item], o.dtype, o.spec, table, tb - 256)
    assert e.value.status == B.GF_ENOMEM
    short = B.gf_batch_item(o.probs[0], o.state.data_ptr(), o.dfom.data_ptr(), o.idx.data_ptr(), o.val.data_ptr(),
                            o.status.data_ptr(), o.fom.data_ptr(), 0, o.ws.data_ptr(), 1024)
    with pytest.raises(B.GfError) as e:
        h.gf_batch_create([short], o.dtype, o.spec, table, tb)
    assert e.value.status == B.GF_ENOMEM
    null_state = B.gf_batch_item(o.probs[0], None, o.dfom.data_ptr(), o.idx.data_ptr(), o.val.data_ptr(),
                                 o.status.data_ptr(), o.fom.data_ptr(), 0, o.ws.data_ptr(), o.ws_bytes)
    with pytest.raises(B.GfError, match="non-NULL"):
        h.gf_batch_create([null_state], o.dtype, o.spec, table, tb)
    b = h.gf_batch_create([item], o.dtype, o.spec, table, tb)
    with pytest.raises(B.GfError):
        h.gf_batch_set_schedule(b, -1)
    for bad in ((7, 0, 1, 32), (B.GF_BATCH_PERSISTENT, -1, 1, 32), (B.GF_BATCH_PERSISTENT, 0, 0, 32),
                (B.GF_BATCH_PERSISTENT, 0, 17, 32), (B.GF_BATCH_PERSISTENT, 0, 1, 48)):
        with pytest.raises(B.GfError) as e:
            h.gf_batch_set_form(b, *bad)
        assert e.value.status == B.GF_EINVAL, bad
    h.gf_batch_set_form(b, B.GF_BATCH_STAGED, 0, 1, 32)
    with pytest.raises(B.GfError):
        h.gf_batch_selftest_timeout(b, 10)            # below the 1 us floor
    h.gf_batch_destroy(b)


def test_c64_batch_against_the_fp64_oracle():
    """The complex64 batch (FP32 stream update, FP64 field and FOM) step by step against the FP64
    oracle directly, not only through the single-problem runs: every problem takes the oracle's
    choices and its G, E and FOM stay within the complex64 tolerance of the oracle's.  The
    monitors sit off the centre line by 0.37 dx, so no mirror-symmetric pair of candidates ties
    exactly (complex64 rounding would otherwise pick either twin)."""
    rng = np.random.default_rng(11)
    wls = []
    for b in range(6):
        side = int(rng.choice([8, 10, 12]))
        wl = W.small(side, side, kind=W.KIND_SINGLE, dir_mask=3, ratio=20,
                     beyond_edge=float(rng.uniform(2.0, 4.0)), steps=4, dtype="c64")
        g = wl.geoms[0]
        g = W.with_monitor(g, g.mon_x + 0.37 * g.dx, g.mon_y)
        wls.append(W.Workload(wl.name, (g,), wl.spec, wl.steps, "c64"))
    bo = BatchOptimizer(wls, dtype="c64")
    bo.fill()
    bo.capture(2)                # one warm-up step runs during capture set-up
    bo.replay()
    torch.cuda.synchronize()
    moved = 0
    for wl, opt in zip(wls, bo.opts):
        orc = O.OracleProblem(wl.geoms, wl.spec)
        for _ in range(3):
            orc.step()
        assert np.array_equal(opt.state.cpu().numpy(), orc.state)
        assert rel_err(opt.G[0][:, :opt.n].cpu().numpy().astype(np.complex128), orc.Gs[0]) <= 2e-5
        assert rel_err(opt.E[0].cpu().numpy(), orc.Es[0]) <= 2e-5
        assert abs(float(opt.fom.cpu()[0]) - orc.fom()) <= 2e-5 * orc.fom()
        moved += int(orc.state.sum())
    assert moved > 0


def test_persistent_step_bounded_wait_reports_timeout():
    """The persistent step's waits are bounded: a diagnostic step whose largest problem waits for
    an evaluation item that does not exist gives up after 20 ms, writes GF_ETIMEOUT to that
    problem's status word and ends; the context stays usable and, refilled, the batch steps
    exactly like the single-problem runs again."""
    wls = _small_batch(4, sides=(8, 10, 12))
    sizes = [w.geoms[0].N for w in wls]
    big = int(np.argmax(sizes))
    bo = BatchOptimizer(wls)
    bo.fill()
    bo._ensure_batches()
    (b,) = bo._batches[0]
    bo.h.gf_batch_selftest_timeout(b, 20_000_000, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert int(bo.opts[big].status.cpu()[0]) == B.GF_ETIMEOUT
    assert float(torch.ones(4, device="cuda").sum().cpu()) == 4.0
    with pytest.raises(B.GfError):
        bo.h.gf_batch_selftest_timeout(b, 10, torch.cuda.current_stream())
    bo.fill()
    bo.capture(2)
    bo.replay()
    torch.cuda.synchronize()
    _check_against_single_runs(wls, bo, 3, "c128", oracle=False)


@pytest.mark.parametrize("sch", [Schedule(0, "given", True), Schedule(0, "given", True, 5), Schedule(3, "given", True),
                                 Schedule(0, "given", True, 0, STAGED), Schedule(0, "given", True, 0, PERSIST, 3)])
def test_tensor_core_batch_update_matches_single_runs_and_oracle(sch):
    """The same small batch with the tensor-core update forced (GF_UPDATE_TENSOR): the persistent
    front launch + the batched tensor-core update + the bands, or the staged launches."""
    wls = _small_batch()
    bo = BatchOptimizer(wls, update_algo=B.GF_UPDATE_TENSOR)
    assert not bo.c128_fma
    bo.schedule = sch
    bo.fill()
    bo.capture(3)
    bo.replay()
    torch.cuda.synchronize()
    _check_against_single_runs(wls, bo, 4, "c128", oracle=True)
