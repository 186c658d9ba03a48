"""Many independent design problems advanced together (the batched pattern of the greedy
step).  Two schedules run the same kernels' arithmetic:

  * fused: the library's batch entry points (up to 64 problems per batch), either as the
    persistent step kernel -- the stages of every problem as work items of one launch, with
    per-problem phase counters (complex128 adds the tensor-core update and the bands as two
    more launches) -- or as one launch per stage of the step;
  * streams: every problem runs its own evaluate / select / update sequence as one branch of
    a fork-join over CUDA streams.

Either way a run of steps is captured once into a CUDA graph and replayed, so launch cost
disappears, and an autotuner picks the schedule (fused: the form, the persistent launch's CTA
count, work-item size and complex64 update tile rows, the update CTAs; streams: a branch count
and order) by timing graph replays.

Nothing here computes: the steps are libgfopt kernels (through the gf_batch_* calls or
GreedyOptimizer).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass
from typing import List, Optional, Sequence

import torch

from . import gfopt as B
from .optimizer import GreedyOptimizer
from .workloads import Workload


@dataclass
class Schedule:
    nstreams: int          # streams: concurrent branches (problems are dealt round-robin onto them)
    order: str             # streams: "given" or "largest_first"
    fused: bool = False    # True: the library's batch entry points; nstreams >= 2 then splits the
                           # problems into that many size-balanced groups on their own streams
    update_ctas: int = 0   # fused: CTAs of the persistent G update (0: the library's default)
    form: int = B.GF_BATCH_PERSISTENT   # fused: persistent step kernel or one launch per stage
    step_ctas: int = 0     # persistent: CTAs (0: all that are resident at once)
    scale: int = 1         # persistent: candidates / rows per thread in one work item
    tile_rows: int = 32    # persistent, complex64: rows of an update tile (16, 32, 64; 0: the
                           # update and the bands as their own launches)


class BatchOptimizer:
    def __init__(self, workloads: Sequence[Workload], dtype: str = "c128", device: int = 0,
                 policies: Optional[Sequence[Optional[tuple]]] = None, horizon: int = 4096,
                 update_algo: Optional[int] = None):
        """policies: per problem None (greedy) or (epsilon, seed) for the epsilon-greedy policy;
        epsilon-greedy batches run on the fused schedule only (its device step counters keep
        drawing new uniforms across graph replays).  update_algo: the G update's arithmetic for
        every schedule (default: the FP64 FMA form where the complex128 batch is small, the sum
        of n^2 p_max within 2.5e6 -- each problem alone then takes that form too -- else the
        tensor-core forms at every size)."""
        self.device = torch.device("cuda", device)
        self.h = B.Handle(device)
        self.workloads = list(workloads)
        # every schedule (fused launches or per-problem stream branches) updates G with the same
        # arithmetic, so that the autotuner's choice of schedule cannot change a single bit of the
        # results
        work = sum((w.geoms[0].N + 1) ** 2 * (1 if w.spec.kind == B.GF_KIND_SINGLE else 4) * max(1, w.spec.k)
                   for w in self.workloads)
        if update_algo is None:
            update_algo = B.GF_UPDATE_TC if (dtype == "c128" and work <= 2.5e6) else B.GF_UPDATE_TENSOR
        self.update_algo = update_algo
        self.c128_fma = dtype == "c128" and (update_algo == B.GF_UPDATE_DFMA or
                                             (update_algo == B.GF_UPDATE_TC and work <= 2.5e6))
        self.h.gf_set_update_algo(update_algo)
        self.opts = [GreedyOptimizer(w.geoms, w.spec, dtype=dtype, device=device, handle=self.h)
                     for w in self.workloads]
        self.policies = list(policies) if policies is not None else [None] * len(self.opts)
        for o, pol in zip(self.opts, self.policies):
            if pol is not None and pol[0] > 0:
                o.set_egreedy(pol[0], seed=pol[1], horizon=horizon)
        self._policy_steps = torch.zeros(len(self.opts), dtype=torch.int32, device=self.device)
        self.exploring = any(o.epsilon is not None for o in self.opts)
        self.sizes = [o.n for o in self.opts]
        self.schedule = Schedule(0, "given", fused=True)
        self._streams: List[torch.cuda.Stream] = []
        self._graph: Optional[torch.cuda.CUDAGraph] = None
        self._graph_steps = 0
        self.applied = torch.zeros(len(self.opts), dtype=torch.int64, device=self.device)
        self._batches = None
        self._batch_groups = 0
        self.fusable = all(o.spec.k == 1 and len(o.geoms) == 1 for o in self.opts)
        if not self.fusable and self.exploring:
            raise ValueError("epsilon-greedy batches need k = 1 and one wavelength per problem")
        if not self.fusable:
            self.schedule = Schedule(min(8, len(self.opts)), "largest_first")

    # ---- the library's batch objects (created on first fused use, per group count)
    def _ensure_batches(self):
        groups = max(1, self.schedule.nstreams)
        if self._batches is not None and self._batch_groups == groups:
            return
        self.close()
        self._applied_step = torch.zeros(len(self.opts), dtype=torch.int32, device=self.device)
        by_size = sorted(range(len(self.opts)), key=lambda i: -self.sizes[i])
        self._batches = []          # list (per group) of gf_batch handles
        self._tables = []
        self._batch_groups = groups
        st = torch.cuda.current_stream(self.device)
        for g in range(groups):
            members = sorted(by_size[g::groups])
            handles = []
            for c0 in range(0, len(members), B.BATCH_MAX):
                items = []
                for i in members[c0:c0 + B.BATCH_MAX]:
                    o = self.opts[i]
                    eps = o.epsilon if o.epsilon is not None else 0.0
                    items.append(B.gf_batch_item(o.probs[0], o.state.data_ptr(), o.dfom.data_ptr(),
                                                 o.idx.data_ptr(), o.val.data_ptr(), o.status.data_ptr(),
                                                 o.fom.data_ptr(), self._applied_step[i:i + 1].data_ptr(),
                                                 o.ws.data_ptr(), o.ws_bytes, eps,
                                                 o._u.data_ptr() if eps > 0 else None,
                                                 self._policy_steps[i:i + 1].data_ptr() if eps > 0 else None,
                                                 int(o._u.shape[0]) if eps > 0 else 0))
                tb = self.h.gf_batch_table_size(len(items))
                table = torch.empty(tb, dtype=torch.uint8, device=self.device)
                self._tables.append(table)
                handles.append(self.h.gf_batch_create(items, self.opts[0].dtype, self.opts[0].spec, table, tb, st))
            if handles:
                self._batches.append(handles)

    def close(self):
        if self._batches:
            for handles in self._batches:
                for b in handles:
                    self.h.gf_batch_destroy(b)
        self._batches = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- set-up
    def fill(self):
        for o in self.opts:
            o.fill()
        self._policy_steps.zero_()
        self.applied.zero_()
        torch.cuda.synchronize(self.device)

    def _order(self) -> List[int]:
        idx = list(range(len(self.opts)))
        if self.schedule.order == "largest_first":
            idx.sort(key=lambda i: -self.sizes[i])
        return idx

    def _ensure_streams(self, count=None):
        while len(self._streams) < (self.schedule.nstreams if count is None else count):
            self._streams.append(torch.cuda.Stream(self.device))

    def _set_form(self, b):
        sch = self.schedule
        self.h.gf_batch_set_schedule(b, sch.update_ctas)
        self.h.gf_batch_set_form(b, sch.form, sch.step_ctas, sch.scale, sch.tile_rows)

    # ---- one step of every problem, enqueued on the current stream
    def enqueue_step(self):
        if self.exploring and not self.schedule.fused:
            raise ValueError("epsilon-greedy batches run on the fused schedule")
        if self.schedule.fused:
            self._ensure_batches()
            main = torch.cuda.current_stream(self.device)
            if len(self._batches) == 1:
                for b in self._batches[0]:
                    self._set_form(b)
                    self.h.gf_batch_step(b, main)
            else:
                self._ensure_streams(len(self._batches))
                start = torch.cuda.Event()
                start.record(main)
                for g, handles in enumerate(self._batches):
                    st = self._streams[g]
                    st.wait_event(start)
                    for b in handles:
                        self._set_form(b)
                        self.h.gf_batch_step(b, st)
                    done = torch.cuda.Event()
                    done.record(st)
                    main.wait_event(done)
            self.applied += self._applied_step
            return
        self._ensure_streams()
        main = torch.cuda.current_stream(self.device)
        start = torch.cuda.Event()
        start.record(main)
        order = self._order()
        lanes = [order[s::self.schedule.nstreams] for s in range(self.schedule.nstreams)]
        for s, lane in enumerate(lanes):
            if not lane:
                continue
            st = self._streams[s]
            st.wait_event(start)
            with torch.cuda.stream(st):
                for i in lane:
                    self.opts[i].step()
                    self.applied[i:i + 1] += self.opts[i].applied.to(torch.int64)
            done = torch.cuda.Event()
            done.record(st)
            main.wait_event(done)

    def capture(self, steps: int) -> torch.cuda.CUDAGraph:
        """Record `steps` batched steps into one CUDA graph (the ops run once during warm-up
        before capture so that every kernel is loaded)."""
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self.enqueue_step()                  # warm-up outside capture
        torch.cuda.current_stream(self.device).wait_stream(side)
        torch.cuda.synchronize(self.device)
        with torch.cuda.graph(g):
            for _ in range(steps):
                self.enqueue_step()
        self._graph = g
        self._graph_steps = steps
        return g

    def replay(self):
        self._graph.replay()

    def autotune(self, candidates: Optional[Sequence[Schedule]] = None, steps: int = 2, reps: int = 2) -> Schedule:
        """Time graph replays of a few schedules and keep the fastest.  Each trial advances the
        problems (the trials are part of the optimisation run)."""
        if candidates is None:
            n = len(self.opts)
            counts = sorted({c for c in (1, 8, 16, n) if c <= n})
            candidates = [Schedule(c, o) for c, o in itertools.product(counts, ("given", "largest_first"))]
            if self.exploring:
                candidates = []
            if self.fusable:
                sms = torch.cuda.get_device_properties(self.device).multi_processor_count
                P = B.GF_BATCH_PERSISTENT
                if self.opts[0].dtype == B.GF_C128:     # one update CTA fits an SM
                    staged = [(1, sms), (2, sms // 2), (2, sms), (4, sms // 4)]
                    persistent = [Schedule(1, "given", True, sms, P, c, s) for c, s in
                                  ((0, 1), (0, 2), (0, 4), (sms, 1))]
                else:
                    staged = [(1, 3 * sms), (1, 6 * sms), (2, 3 * sms), (4, 3 * sms)]
                    persistent = [Schedule(1, "given", True, u, P, c, s, r) for u, c, s, r in
                                  ((0, 0, 1, 64), (0, 0, 2, 64), (0, 0, 1, 32), (3 * sms, 0, 1, 0),
                                   (6 * sms, 0, 1, 0), (3 * sms, 0, 4, 0))]
                candidates = persistent + [Schedule(g, "given", True, c, B.GF_BATCH_STAGED)
                                           for g, c in staged] + candidates
        best, best_ms = None, float("inf")
        self.timings = []
        for sch in candidates:
            self.schedule = sch
            self.capture(steps)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            self.replay()
            torch.cuda.synchronize(self.device)
            e0.record()
            for _ in range(reps):
                self.replay()
            e1.record()
            torch.cuda.synchronize(self.device)
            ms = e0.elapsed_time(e1) / (reps * steps)
            self.timings.append((sch, ms))
            if ms < best_ms:
                best, best_ms = sch, ms
        self.schedule = best
        self._graph = None
        return best

    def total_applied(self) -> int:
        return int(self.applied.sum().item())
