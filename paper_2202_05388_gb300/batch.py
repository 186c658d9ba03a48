"""Many independent design problems advanced together (the batched pattern of the greedy
step): every problem runs its own evaluate / select / update sequence as one branch of a
fork-join over CUDA streams, and a whole run of steps is captured once into a CUDA graph and
replayed, so the per-kernel launch cost of the small problems disappears and the problems'
kernels overlap on the GPU.  An autotuner picks the number of concurrent branches and their
order by timing graph replays.

Nothing here computes: the steps are the libgfopt kernels driven through GreedyOptimizer.
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
    nstreams: int          # concurrent branches (problems are dealt round-robin onto them)
    order: str             # "given" or "largest_first"


class BatchOptimizer:
    def __init__(self, workloads: Sequence[Workload], dtype: str = "c128", device: int = 0):
        self.device = torch.device("cuda", device)
        self.h = B.Handle(device)
        self.workloads = list(workloads)
        self.opts = [GreedyOptimizer(w.geoms, w.spec, dtype=dtype, device=device, handle=self.h)
                     for w in self.workloads]
        self.sizes = [o.n for o in self.opts]
        self.schedule = Schedule(min(8, len(self.opts)), "largest_first")
        self._streams: List[torch.cuda.Stream] = []
        self._graph: Optional[torch.cuda.CUDAGraph] = None
        self._graph_steps = 0
        self.applied = torch.zeros(len(self.opts), dtype=torch.int64, device=self.device)

    # ---- set-up
    def fill(self):
        for o in self.opts:
            o.fill()
        torch.cuda.synchronize(self.device)

    def _order(self) -> List[int]:
        idx = list(range(len(self.opts)))
        if self.schedule.order == "largest_first":
            idx.sort(key=lambda i: -self.sizes[i])
        return idx

    def _ensure_streams(self):
        while len(self._streams) < self.schedule.nstreams:
            self._streams.append(torch.cuda.Stream(self.device))

    # ---- one step of every problem, enqueued as a fork-join on the current stream
    def enqueue_step(self):
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
            counts = sorted({c for c in (1, 4, 8, 16, n) if c <= n})
            candidates = [Schedule(c, o) for c, o in itertools.product(counts, ("given", "largest_first"))]
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
