"""Throughput of the greedy Green's-function optimizer step on GB300.

A step is one pass of the whole hot path on the 192x192 2x2-brush workload with a
complex128 G (N = 36864 pixels, n = N+1 = 36865, 72962 candidates, G = 21.7 GB):
evaluate every candidate's exact dFOM, select the best, and apply the rank-p update to G
and E.  The metric is accepted flips per second (one accepted brush per step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

--impl reference times the FP64 CPU oracle on the host cores instead (each step a bounded
row/candidate sample of the same workload, scaled to a full step).  Under torchrun every rank
runs an independent replica of the problem (the path has no exchange step on one GPU);
value = flips of all ranks / max wall time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

from paper_2202_05388_gb300 import workloads as W

METRIC = "accepted flips/s (greedy step: dFOM of every 2x2 brush + select + rank-p G/E update)"
UNIT = "flips/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default="brush_192")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-breakdown", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work")
    ap.add_argument("--graph", action="store_true",
                    help="capture the K timed steps in one CUDA graph and time its replay")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-precision vs FP64 comparison on the 320x320 geometry")
    ap.add_argument("--mixed-err-steps", type=int, default=3,
                    help="lock-step steps of the mixed form's error statement against the FP64 path")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--replicas", action="store_true",
                    help="with several ranks: independent replicas instead of one problem split by rows")
    ap.add_argument("--update-algo", choices=["tc", "dfma", "tensor"], default="tc",
                    help="arithmetic of the G update (gf_set_update_algo): the fastest form per case "
                         "(default), FP64 FMA, or the tensor-core forms at every size")
    return ap.parse_args()


def workload(name):
    return {"brush_192": W.brush_192, "plain_32": W.plain_32, "brush_64": W.brush_64, "brush_128": W.brush_128,
            "brush_128_topk": W.brush_128_topk, "brush_320_c128": W.brush_320_c128,
            "brush_320_c64_rank4": W.brush_320_c64_rank4, "brush_96_c64_rank4": W.brush_96_c64_rank4,
            "brush_320_topk": W.brush_320_topk, "multilambda_512x64": W.multi_lambda_512x64}[name]()


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                pw.append(float(r[3]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one update launch, from a
# single-pass ncu capture of the same kernel on the 128x128 member of the workload's family
# (G = 4.3 GB, 33x the L2), scaled to the full-size launch by the entries updated (n^2); valid
# only for the kernel source it was taken on (SHA-256 over the files below), otherwise null.
TRAFFIC_SOURCES = ("paper_2202_05388_gb300/csrc/gf_update_tc.cu", "paper_2202_05388_gb300/csrc/gf_tc.cuh")
TRAFFIC = {
    "brush_192x192_p4_c128": {"sha256": "fbd391f1ecb93c65d7da81de0c34bb3324ec1789146d47ad4e298ba945b261e3",
                              "capture_n": 16385, "capture_bytes": 4.3094e9 + 4.2393e9, "n": 36865,
                              "profile": "profiles/rank_update_tc_brush128_traffic.md"},
}


def measured_traffic(workload_name):
    import hashlib
    rec = TRAFFIC.get(workload_name)
    if rec is None:
        return None
    h = hashlib.sha256()
    root = os.path.dirname(os.path.abspath(__file__))
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(root, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != rec["sha256"]:
        return None
    return rec["capture_bytes"] * (rec["n"] / rec["capture_n"]) ** 2


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def f16_peak_tflops():
    """Dense FP16 tensor peak: the measured BF16 burst peak x the nominal FP16/BF16 ratio (1)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d.get("bf16_tflops", 1900.0), "measured bf16 burst x nominal fp16/bf16 (1.0)"
    return 1900.0, "fallback bf16 x nominal fp16/bf16 (1.0)"


# FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (unit count x max clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


# ------------------------------------------------------------------------------ CPU oracle
def oracle_step_sample(wl, budget_s, rng_seed=0):
    """Time the FP64 oracle on a bounded sample of one greedy step of workload `wl` and scale
    it to a full step.  Sample: (a) every candidate of a strip of image rows of the design
    (the oracle's vectorised evaluation on a sub-grid with the same nx, dx and monitor),
    scaled by the candidate count; (b) the oracle's Eq. 10 row update on a block of rows of
    the full n x n G, scaled by n / rows.  Returns (seconds per full step, description)."""
    from oracle import gf_oracle as O
    g = wl.geoms[0]
    spec = wl.spec
    n = g.N + 1
    # (a) candidate evaluation on a strip of `sy` image rows (same nx, dx, monitor)
    sy = 6
    gs = W.Geometry(g.nx, sy, g.dx, g.wavelength, g.mon_x, g.mon_y, g.eps_bg, g.eps_mat)
    strip = O.OracleProblem([gs], spec)
    t0 = time.perf_counter()
    d = strip.evaluate()
    t_eval = time.perf_counter() - t0
    ncand_strip = d.size
    ncand_full = O.num_candidates(g, spec)
    eval_full = t_eval * ncand_full / ncand_strip
    # (b) Eq. 10 on a row block of the full G (rows built from G0, p = 4 columns)
    rng = np.random.default_rng(rng_seed)
    p = 4 if spec.kind == W.KIND_BRUSH2 else 1
    pts = O.points(g)
    rows = 256
    V = rng.choice(g.N, size=p, replace=False)

    def g0_rows(r0, r1):
        d2 = pts[r0:r1, None, :] - pts[None, :, :]
        r = np.sqrt(d2[..., 0] ** 2 + d2[..., 1] ** 2)
        with np.errstate(divide="ignore", invalid="ignore"):
            M = O.g0_pair(g, r)
        for i in range(r0, r1):
            if i < g.N:
                M[i - r0, i] = O.g0_self(g)
            else:
                M[i - r0, i] = 0.0
        return M

    Grows = g0_rows(0, rows)
    R = g0_rows(0, p)                    # stands in for A^{-1} G[V, :] (same shape and scale)
    C = Grows[:, V].copy()
    dchi = np.full(p, g.eps_mat - g.eps_bg)
    reps, t_upd = 0, 0.0
    while t_upd < 0.5 * budget_s and reps < 64:
        t0 = time.perf_counter()
        _ = O.update_rows(Grows, C, dchi, R)
        t_upd += time.perf_counter() - t0
        reps += 1
    upd_full = (t_upd / reps) * n / rows
    # (c) selection over all candidates
    dd = np.random.default_rng(1).normal(size=ncand_full)
    t0 = time.perf_counter()
    _ = O.select_best(dd, spec.tie_rel)
    t_sel = time.perf_counter() - t0
    step = eval_full + upd_full + t_sel
    desc = (f"oracle dFOM of all {ncand_strip} candidates of a {g.nx}x{sy} strip scaled x"
            f"{ncand_full / ncand_strip:.1f}; Eq. 10 update of {rows} of {n} rows (x{reps}) scaled "
            f"x{n / rows:.0f}; selection over {ncand_full}")
    return step, desc, {"eval_s": eval_full, "update_s": upd_full, "select_s": t_sel}


def blas_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] or [1])
    except Exception:
        return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


SINGLE_THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def oracle_sample_single_thread(wl_name, budget_s):
    """The same bounded oracle sample in a child process whose BLAS runs one thread (the
    thread count of numpy's BLAS is fixed when it loads, so it takes a fresh process)."""
    env = dict(os.environ)
    for k in SINGLE_THREAD_ENV:
        env[k] = "1"
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", f"{wl_name}:{budget_s}"],
                       env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(wl, budget_s, wl_name="brush_192"):
    step, desc, parts = oracle_step_sample(wl, budget_s)
    out = {"value": 1.0 / step, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
           "sample": desc, "seconds_per_step": step, "parts_s": parts}
    one = oracle_sample_single_thread(wl_name, max(2.0, budget_s / 2))
    if one is not None:
        out["single_thread"] = {"value": 1.0 / one["seconds_per_step"], "unit": UNIT, "cores": 1,
                                "seconds_per_step": one["seconds_per_step"], "parts_s": one["parts_s"],
                                "note": "same sample, BLAS limited to one thread in a child process"}
    return out


# ------------------------------------------------------------------------------ dist
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_replicas(ms: float, flips: int, device) -> tuple:
    """Across the ranks of the initialised process group: the slowest rank's time and the
    flips of all ranks (every rank runs its own replica; no data path crosses ranks)."""
    import torch
    import torch.distributed as dist
    tt = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ff = torch.tensor([flips], dtype=torch.int64, device=device)
    dist.all_reduce(ff)
    return float(tt.item()), int(ff.item())


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    wl = workload(args.workload)
    for _ in range(args.warmup):
        oracle_step_sample(wl, 2.0)
    times = []
    desc = ""
    for _ in range(args.steps):
        s, desc, _ = oracle_step_sample(wl, 2.0)
        times.append(s)
    total = sum(times)
    value = args.steps / total
    g = wl.geoms[0]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "nx": g.nx, "ny": g.ny, "n": g.N + 1,
                       "candidates": W.CandidateSpec(wl.spec.kind, wl.spec.dir_mask).ncand(g)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ native
def sched_json(s):
    from paper_2202_05388_gb300 import gfopt as B
    if s.fused:
        out = {"fused": True, "groups": max(1, s.nstreams), "update_ctas": s.update_ctas or "default"}
        if s.form == B.GF_BATCH_PERSISTENT:
            out.update({"form": "persistent", "step_ctas": s.step_ctas or "all resident", "scale": s.scale,
                        "tile_rows": s.tile_rows or "update as its own launch"})
        else:
            out["form"] = "staged"
        return out
    return {"fused": False, "streams": s.nstreams, "order": s.order}


def persistent_single_problem(wl, args):
    """The same problem as a batch of one on the persistent step kernel (for a small complex128
    problem the whole step, FP64 FMA update included, is one launch), K steps in one CUDA graph
    after W steps from the filled start: the per-step cost without the stage launches."""
    import torch
    from paper_2202_05388_gb300 import gfopt as B
    from paper_2202_05388_gb300.batch import BatchOptimizer, Schedule
    bo = BatchOptimizer([wl], dtype=wl.dtype)
    bo.schedule = Schedule(0, "given", True, 0, B.GF_BATCH_PERSISTENT)
    bo.fill()
    for _ in range(max(0, args.warmup - 1)):
        bo.enqueue_step()
    bo.capture(args.steps)                    # one more step runs before the capture
    before = bo.total_applied()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    bo.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out = {"ms_per_step": ms / args.steps, "steps_per_s": args.steps / (ms / 1e3),
           "accepted_flips": bo.total_applied() - before,
           "launches_per_step": 1 if (bo.c128_fma or wl.dtype == "c64") else 3,
           "update": "FP64 FMA" if bo.c128_fma else ("FP32 stream" if wl.dtype == "c64" else "tensor cores")}
    bo.close()
    return out


def select_launches(ncand):
    """Launches of the greedy (k = 1) selection with a workspace: one CTA, or from 32768
    candidates a pass over many CTAs and a finishing CTA."""
    return 2 if ncand >= 32768 else 1


def launches_per_step(s, nprob, dtype, c128_fma=False):
    """Library kernels per batched step, per group of 64 problems: persistent = the step kernel
    (complex128, or complex64 with tile_rows 0: + the G update and the bands); staged = one launch per stage (eval,
    select, capacitance, panels, [digit prep], update, finish, bands); stream branches = the
    single-problem sequence per problem (eval, select, capacitance, panels, [2 digit preps],
    update, finish, bands)."""
    from paper_2202_05388_gb300 import gfopt as B
    if s.fused:
        groups = max(1, s.nstreams)
        per_group = -(-nprob // groups)
        if s.form == B.GF_BATCH_PERSISTENT:
            per = 3 if ((dtype == "c128" and not c128_fma) or (dtype != "c128" and s.tile_rows == 0)) else 1
        else:
            per = 8 if (dtype == "c128" and not c128_fma) else 7
        return groups * ((per_group + 63) // 64) * per
    return nprob * (9 if dtype == "c128" else 7)


def run_batch(args):
    """48 independent single-pixel problems (seeded sizes) advanced together: autotuned
    schedule (fused batch launches or fork-join stream branches), K steps captured in one CUDA
    graph and replayed in the timed region."""
    import torch
    from paper_2202_05388_gb300 import build as BLD
    from paper_2202_05388_gb300.batch import BatchOptimizer

    from paper_2202_05388_gb300 import gfopt as B

    torch.cuda.set_device(0)
    BLD.build()
    dtype = "c64" if args.workload.endswith("c64") else "c128"
    wls = W.batch_48()
    bo = BatchOptimizer(wls, dtype=dtype)
    bo.fill()
    best = bo.autotune(steps=1, reps=1)

    def timed_run(sch, clocks=None):
        """From the filled start: warm-up replay of K steps, then one timed replay of K steps."""
        bo.fill()
        bo.schedule = sch
        bo.capture(args.steps)
        bo.replay()                               # warm-up replay
        torch.cuda.synchronize()
        before = bo.total_applied()
        if clocks is not None:
            clocks.start()
            time.sleep(0.3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bo.replay()
        e1.record()
        torch.cuda.synchronize()
        clk = clocks.stop() if clocks is not None else None
        return e0.elapsed_time(e1), bo.total_applied() - before, clk

    # the best schedule of each fused form, timed on the same trajectory (both forms give
    # bit-identical results, so the work is the same)
    forms = {}
    for name, code in (("persistent", B.GF_BATCH_PERSISTENT), ("staged", B.GF_BATCH_STAGED)):
        tried = [t for t in bo.timings if t[0].fused and t[0].form == code]
        if tried:
            sch = min(tried, key=lambda t: t[1])[0]
            fms, fflips, _ = timed_run(sch)
            forms[name] = {"schedule": sched_json(sch), "ms_per_step": fms / args.steps, "accepted_flips": fflips}
    ms, flips, clk = timed_run(best, ClockSampler(0))
    sumG = sum(o.G[0].numel() * o.G[0].element_size() for o in bo.opts)
    bytes_step = sum(o.n * o.n for o in bo.opts) * (32 if dtype == "c128" else 16)
    peak_hbm, peak_kind = measured_peaks()
    gbs = bytes_step * args.steps / (ms * 1e-3) / 1e9
    line = {"metric": METRIC + " [48 batched problems]", "value": flips / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if dtype == "c128" else "f32",
            "data": "synthetic",
            "config": {"workload": f"batch48_single_pixel_{dtype}", "problems": len(wls), "sum_G_GB": sumG / 1e9,
                       "storage": dtype, "schedule": sched_json(best),
                       "autotune_ms_per_step": [[sched_json(t[0]), t[1]] for t in bo.timings],
                       "fused_forms": forms,
                       "graph": f"{args.steps} steps of all problems in one CUDA graph",
                       "l2": "inputs larger than L2 (sum of G %.1f GB)" % (sumG / 1e9)},
            "accepted_flips": flips,
            "gpu_launches": launches_per_step(best, len(wls), dtype, bo.c128_fma) * args.steps,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak_hbm, "unit": "GB/s", "frac": gbs / peak_hbm,
                         "traffic": None, "peak_kind": peak_kind,
                         "note": "whole step (all kernels of all problems): algorithmic G bytes / step time"},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def mixed_comparison(K, err_steps, dev):
    """The mixed-precision form against the plain FP64 form on one geometry (320x320 pixels,
    dx = lambda/20, focus 5 lambda past the far edge), both timed over steps 1..K from the vacuum
    start (fill excluded): complex64 G with the top-32 rank-k p Woodbury update, and complex128 G
    with one brush (rank 4) per step.  Then the error statement: the complex64 form and the
    library's complex128 path run lock-step on the complex64 form's own choices for err_steps
    steps from vacuum (the complex128 path applies the same ids; it matches the FP64 oracle
    within 1e-10 in the parity tests), comparing E, the FOM and 4096 sampled G entries after
    every step.  Each G is freed before the next one is allocated, except the two of the
    lock-step run (84 + 168 GB)."""
    import gc
    import torch
    from paper_2202_05388_gb300.optimizer import GreedyOptimizer

    peak_hbm, peak_kind = measured_peaks()

    def free():
        gc.collect()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    def timed(wl):
        opt = GreedyOptimizer(wl.geoms, wl.spec, dtype=wl.dtype, device=dev)
        opt.fill()
        acc = torch.zeros(1, dtype=torch.int64, device=f"cuda:{dev}")
        torch.cuda.synchronize()
        opt.h.gf_profile_begin(K + 4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            opt.step()
            acc += opt.applied.to(torch.int64)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kms, kn, kb, _ = opt.h.gf_profile_end()
        flips = int(acc.item())
        gbs = (kb / kn) / (kms / kn * 1e-3) / 1e9 if kn else 0.0
        return opt, {"flips_per_s": flips / (ms / 1e3), "ms_per_step": ms / K, "accepted_flips": flips,
                     "update_ms_avg": kms / max(kn, 1), "update_GBps": gbs, "update_frac": gbs / peak_hbm,
                     "update_launches": kn}

    wl64, wl128 = W.brush_320_topk(), W.brush_320_c128()
    # load every kernel of the complex64 top-k path first (both update forms) on a small member
    warm = GreedyOptimizer(W.brush_128_topk().geoms, W.brush_128_topk().spec, dtype="c64", device=dev)
    warm.fill()
    for _ in range(3):
        warm.step()
    del warm
    free()
    o128, r128 = timed(wl128)
    del o128
    free()
    o64, r64 = timed(wl64)
    # error statement: lock-step from vacuum against the complex128 path on the same choices
    o64.fill()
    ref = GreedyOptimizer(wl64.geoms, wl64.spec, dtype="c128", device=dev)
    ref.fill()
    n = wl64.geoms[0].N + 1
    rng = np.random.default_rng(5)
    ri = torch.tensor(rng.integers(0, n, 4096), device=f"cuda:{dev}")
    ci = torch.tensor(rng.integers(0, n, 4096), device=f"cuda:{dev}")
    per_step = []
    t0 = time.perf_counter()
    for t in range(err_steps):
        o64.step()
        ref.idx.copy_(o64.idx)
        ref.status.copy_(o64.status)
        ref.update()
        torch.cuda.synchronize()
        g64 = o64.G[0][ri, ci].to(torch.complex128)
        g128 = ref.G[0][ri, ci]
        eG = float((g64 - g128).abs().max() / g128.abs().max())
        eE = float((o64.E[0] - ref.E[0]).abs().max() / ref.E[0].abs().max())
        f64, f128 = float(o64.fom.cpu()[0]), float(ref.fom.cpu()[0])
        same = bool(torch.equal(o64.state, ref.state))
        per_step.append({"step": t + 1, "applied": int(o64.applied.cpu()[0]), "G_sampled_rel": eG, "E_rel": eE,
                         "FOM_rel": abs(f64 - f128) / f128, "same_decision": same})
    err_s = time.perf_counter() - t0
    del o64, ref
    free()
    return {"workload": wl64.name, "fp64_workload": wl128.name, "window": f"steps 1..{K} from the vacuum start "
            "(fill excluded), K CUDA-event-timed eager steps", "mixed": r64, "fp64": r128,
            "flips_ratio_mixed_over_fp64": r64["flips_per_s"] / r128["flips_per_s"],
            "peak_kind": peak_kind,
            "error_vs_fp64": {"steps": err_steps, "per_step": per_step,
                              "G_sampled_rel_max": max(x["G_sampled_rel"] for x in per_step),
                              "E_rel_max": max(x["E_rel"] for x in per_step),
                              "FOM_rel_max": max(x["FOM_rel"] for x in per_step),
                              "reference": "the library's complex128 path applying the complex64 form's choices "
                                           "(within 1e-10 of the FP64 oracle in the parity tests)",
                              "metric": "max-norm relative: max |x64 - x128| / max |x128| over 4096 seeded G "
                                        "entries, all of E; |FOM64 - FOM128| / FOM128",
                              "seconds": err_s}}


def run_sharded(args):
    """One problem split by rows over the ranks (paper Sec. III's partitions, one per GPU): every
    step evaluates each rank's candidates, takes the elementwise max of the dFOM arrays, selects,
    sums the row panels of the update set (the owners' broadcast) and updates each rank's rows.
    value = the problem's accepted flips / the slowest rank's time (strong scaling: the total work
    is fixed).  Collectives over NCCL; GF_BENCH_BACKEND=gloo runs the ranks on the GPUs available
    (rank r on device r mod count), which lets two ranks share one GPU for a check."""
    import torch
    import torch.distributed as dist
    from paper_2202_05388_gb300 import build as BLD
    from paper_2202_05388_gb300 import gfopt as B
    from paper_2202_05388_gb300.sharded import ShardedOptimizer

    rank, world, local = dist_env()
    backend = os.environ.get("GF_BENCH_BACKEND", "nccl")
    dev = local % max(1, torch.cuda.device_count())
    torch.cuda.set_device(dev)
    dist.init_process_group(backend)
    if rank == 0:
        BLD.build()
    dist.barrier()
    wl = workload(args.workload)
    g = wl.geoms[0]
    opt = ShardedOptimizer(g, wl.spec, dtype=wl.dtype, device=dev)
    sh = opt.shard
    opt.fill()
    acc = torch.zeros(1, dtype=torch.int64, device=f"cuda:{dev}")
    for _ in range(args.warmup):
        opt.step()
        acc += sh.applied.to(torch.int64)
    acc.zero_()
    torch.cuda.synchronize()
    dist.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    sh.h.gf_profile_begin(args.steps + 4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        opt.step()
        acc += sh.applied.to(torch.int64)
    e1.record()
    torch.cuda.synchronize()
    dist.barrier()
    ms = e0.elapsed_time(e1)
    kms, kn, kb, _ = sh.h.gf_profile_end()
    clk = clocks.stop()
    flips = int(acc.item())                       # the same on every rank: one problem
    tt = torch.tensor([ms], dtype=torch.float64, device=f"cuda:{dev}")
    if backend == "gloo":
        tt = tt.cpu()
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    t_max = float(tt.item())
    # end to end through the sharded optimizer: H2D of the design state, K steps each with a D2H of the step record
    host_state = torch.zeros(g.N, dtype=torch.uint8).pin_memory()
    rec = sh.step_record()
    host_rec = torch.empty(rec.numel(), dtype=torch.float64).pin_memory()
    opt.fill()
    dist.barrier()
    t0 = time.perf_counter()
    sh.state.copy_(host_state, non_blocking=True)
    done = 0
    for _ in range(args.steps):
        opt.step()
        host_rec.copy_(sh.step_record(), non_blocking=True)
        torch.cuda.current_stream().synchronize()
        done += int(host_rec[-1].item())
    t_e2e = time.perf_counter() - t0
    te = torch.tensor([t_e2e], dtype=torch.float64)
    if backend != "gloo":
        te = te.to(f"cuda:{dev}")
    dist.all_reduce(te, op=dist.ReduceOp.MAX)
    t_e2e = float(te.item())
    if rank == 0:
        peak_hbm, peak_kind = measured_peaks()
        bpl = kb / max(kn, 1)
        kavg = kms / max(kn, 1)
        gbs = bpl / (kavg * 1e-3) / 1e9 if kavg > 0 else 0.0
        panel_bytes = sh.pmax * sh.ldg * (16 if wl.dtype == "c128" else 8)
        line = {"metric": METRIC, "value": flips / (t_max / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f64" if wl.dtype == "c128" else "f32",
                "data": "synthetic",
                "config": {"workload": wl.name, "nx": g.nx, "ny": g.ny, "n": g.N + 1,
                           "parallelism": f"row shards x{world} ({backend})",
                           "pixel_rows_per_rank": [b[1] - b[0] for b in opt.bands_of_rank],
                           "G_rows_rank0": sh.rows, "l2": "inputs larger than L2",
                           "exchange_bytes_per_step": {"dfom_max": sh.ncand * 8, "row_panel_sum": panel_bytes,
                                                       "halo_allgather": (B.GF_NBANDS + 1) * g.nx * 16 * world}},
                "accepted_flips": flips,
                "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak_hbm, "unit": "GB/s",
                             "frac": gbs / peak_hbm, "traffic": None, "peak_kind": peak_kind,
                             "kernel": "rank 0's row-block update (k_rank_update_ozaki on its rows)",
                             "kernel_ms_avg": kavg, "algorithmic_bytes_per_launch": bpl},
                # per step on each rank: -inf fill + dFOM, selection, row gather, capacitance, panels,
                # the update's launches (digit preparation of rows and columns + the tensor-core
                # update, or one FP64 FMA launch), field/FOM, band read-back, halo pack and unpack
                "gpu_launches": args.steps * (9 + select_launches(sh.ncand) +
                                              (3 if wl.dtype == "c128" and wl.spec.k == 1 else 1)),
                "clocks": clk,
                "e2e": {"value": done / t_e2e, "unit": UNIT, "h2d_bytes_per_step": g.N / args.steps,
                        "d2h_bytes_per_step": host_rec.numel() * 8,
                        "note": "timed: H2D of the design state, then K x (sharded step + D2H of the step record)"}}
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()
    return 0


def run_native(args):
    import torch
    from paper_2202_05388_gb300 import build as BLD
    from paper_2202_05388_gb300 import gfopt as B
    from paper_2202_05388_gb300.optimizer import GreedyOptimizer

    rank, world, local = dist_env()
    if world > 1 and not args.replicas:
        return run_sharded(args)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    if rank == 0:
        BLD.build()
    if world > 1:
        torch.distributed.barrier()
    wl = workload(args.workload)
    g = wl.geoms[0]
    opt = GreedyOptimizer(wl.geoms, wl.spec, dtype=wl.dtype, device=dev)
    if args.update_algo != "tc":
        opt.h.gf_set_update_algo(B.GF_UPDATE_DFMA if args.update_algo == "dfma" else B.GF_UPDATE_TENSOR)
    opt.fill()
    torch.cuda.synchronize()
    accepted = torch.zeros(1, dtype=torch.int64, device=f"cuda:{dev}")
    # warm-up runs exactly the timed loop body, so that every kernel (ours and torch's
    # bookkeeping ops) is loaded before timing -- lazy module loading costs seconds
    for _ in range(args.warmup):
        opt.step()
        accepted += opt.applied.to(torch.int64)
    accepted.zero_()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    nlam = len(wl.geoms)
    if args.graph:
        # the K steps captured once into a CUDA graph (launch cost leaves the timed region);
        # the update kernel's own time comes from an eager pass after the timed replay
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(args.steps):
                opt.step()
                accepted += opt.applied.to(torch.int64)
        torch.cuda.synchronize()
        accepted.zero_()
        torch.cuda.synchronize()
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        opt.h.gf_profile_begin(args.steps * nlam + 4)
        for _ in range(args.steps):
            opt.step()
        kern_ms, kern_launches, kern_bytes, kern_flops = opt.h.gf_profile_end()
        persistent_one = persistent_single_problem(wl, args) if (nlam == 1 and wl.spec.k == 1) else None
    else:
        opt.h.gf_profile_begin(args.steps * nlam + 4)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            opt.step()
            accepted += opt.applied.to(torch.int64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kern_ms, kern_launches, kern_bytes, kern_flops = opt.h.gf_profile_end()
    clk = clocks.stop()
    flips = int(accepted.item())
    t_max = ms
    flips_total = flips
    if world > 1:
        t_max, flips_total = reduce_replicas(ms, flips, f"cuda:{dev}")
    value = flips_total / (t_max / 1e3)

    # ---- per-stage breakdown (CUDA events around each ABI call; not part of the timed region)
    breakdown = None
    dfma = None
    if not args.no_breakdown:
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        parts = {"eval": 0.0, "select": 0.0, "update": 0.0}
        nb = 3
        for _ in range(nb):
            evs[0].record(stream)
            opt.evaluate()
            evs[1].record(stream)
            opt.select()
            evs[2].record(stream)
            opt.update()
            evs[3].record(stream)
            torch.cuda.synchronize()
            parts["eval"] += evs[0].elapsed_time(evs[1]) / nb
            parts["select"] += evs[1].elapsed_time(evs[2]) / nb
            parts["update"] += evs[2].elapsed_time(evs[3]) / nb
        breakdown = parts
        if wl.dtype == "c128":
            opt.h.gf_set_update_algo(B.GF_UPDATE_DFMA)
            opt.h.gf_profile_begin(8)
            for _ in range(2):
                opt.step()
            torch.cuda.synchronize()
            d_ms, d_n, d_b, d_f = opt.h.gf_profile_end()
            opt.h.gf_set_update_algo(B.GF_UPDATE_TC)
            if d_n:
                dfma = {"kernel": "k_rank_update_f64 (native DFMA)", "ms": d_ms / d_n,
                        "tflops": d_f / d_n / (d_ms / d_n * 1e-3) / 1e12,
                        "fp64_peak_tflops": FP64_PEAK_TFLOPS,
                        "GBps": d_b / d_n / (d_ms / d_n * 1e-3) / 1e9}

    # ---- end to end through the public API: host input -> device -> K steps -> host results
    e2e = None
    if not args.no_e2e:
        host_state = torch.zeros(g.N, dtype=torch.uint8).pin_memory()
        k = max(1, wl.spec.k)
        # two pinned result buffers: step t's result is read once step t + 1 is enqueued, so the
        # host's launches of a step overlap the GPU's work on the previous one (a step after the
        # last improving one is a no-op on the device, as the status word makes it)
        host_out = [torch.empty(2 * k + 3, dtype=torch.float64).pin_memory() for _ in range(2)]
        done_ev = [torch.cuda.Event(), torch.cuda.Event()]
        opt2 = opt

        def e2e_enqueue(slot):
            opt2.step()
            packed = torch.cat([opt2.idx[:k].to(torch.float64), opt2.val[:k],
                                opt2.status.to(torch.float64), opt2.fom, opt2.applied.to(torch.float64)])
            host_out[slot].copy_(packed, non_blocking=True)
            done_ev[slot].record()

        def e2e_read(slot):
            done_ev[slot].synchronize()
            return int(host_out[slot][2 * k + 2].item())

        def e2e_run(nsteps):
            acc = 0
            for t in range(nsteps):
                e2e_enqueue(t % 2)
                if t > 0:
                    acc += e2e_read((t - 1) % 2)
            return acc + (e2e_read((nsteps - 1) % 2) if nsteps > 0 else 0)

        opt2.state.copy_(host_state, non_blocking=True)
        opt2.fill()
        e2e_run(2)                  # warm-up of the same body (module loading, allocator)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        opt2.state.copy_(host_state, non_blocking=True)       # job input: the design state
        opt2.fill()
        acc2 = e2e_run(args.steps)
        t_e2e = time.perf_counter() - t0
        e2e = {"value": acc2 / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": g.N / args.steps,
               "d2h_bytes_per_step": host_out[0].numel() * 8,
               "note": "timed: H2D of the design state, gf_fill_g0, then K x (step + D2H of "
                       "the step result) through GreedyOptimizer; step t's result is read from "
                       "pinned memory after step t + 1 is enqueued"}

    # ---- drift refresh (every few hundred steps in a run; timed once here, outside the step)
    refresh = None
    if not args.no_breakdown:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rr = opt.refresh(nsample=8, tol=1e-12 if wl.dtype == "c128" else 1e-8)
        refresh = {"ms": 1e3 * (time.perf_counter() - t0), "ls_residual": rr[0][0][0],
                   "column_drift_max": max(rr[0][0][1:]) if len(rr[0][0]) > 1 else None,
                   "column_residual_max": max(rr[0][2]) if rr[0][2] else None,
                   "gmres_iters": rr[0][1], "columns": 8,
                   "note": "column_drift: stored column vs its GMRES re-solve (0 when the stored column "
                           "already meets the tolerance); column_residual: the stored column's own Eq. 2 "
                           "residual (backward error)"}

    ncand_main, G_GB_main = opt.ncand, opt.G[0].numel() * opt.G[0].element_size() / 1e9
    mixed = None
    if rank == 0 and world == 1 and args.workload == "brush_192" and not args.no_mixed:
        # the dense 192x192 problem is freed first: the comparison needs up to 252 GB of HBM
        opt2 = None
        del opt
        mixed = mixed_comparison(args.steps, args.mixed_err_steps, dev)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    peak_hbm, peak_kind = measured_peaks()
    kern_avg_ms = kern_ms / max(kern_launches, 1)
    bytes_per_launch = kern_bytes / max(kern_launches, 1)
    flops_per_launch = kern_flops / max(kern_launches, 1)
    achieved_gbs = bytes_per_launch / (kern_avg_ms * 1e-3) / 1e9
    achieved_tfl = flops_per_launch / (kern_avg_ms * 1e-3) / 1e12
    pmax_upd = wl.spec.k * (4 if wl.spec.kind == 1 else 1)
    n_upd = g.N + 1
    oz = wl.dtype == "c128" and pmax_upd <= 4 and (
        args.update_algo == "tensor" or (args.update_algo == "tc" and n_upd * n_upd * pmax_upd > 2.5e6))
    if wl.dtype == "c128" and not oz:
        # the FP64 FMA kernel: the library's choice for L2-resident problems (n^2 p_max <= 2.5e6)
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": peak_hbm, "unit": "GB/s",
                "frac": achieved_gbs / peak_hbm, "traffic": None, "peak_kind": peak_kind,
                "kernel": "k_rank_update_f64 (FP64 FMA)",
                "note": "G is L2-resident at this size: the launch is latency-bound, not HBM-bound"
                        if n_upd * n_upd * 16 < 64e6 else "FP64-pipe bound"}
    elif wl.dtype == "c128":
        tr = measured_traffic(wl.name)
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": peak_hbm, "unit": "GB/s",
                "frac": achieved_gbs / peak_hbm, "traffic": tr, "peak_kind": peak_kind,
                "traffic_note": "bytes per launch: ncu capture of this kernel on the 128x128 member of the workload "
                                "family (4.3 GB), scaled by n^2 to this size; kernel source unchanged since"
                                if tr is not None else "no capture for this workload / kernel source",
                "kernel": "k_rank_update_ozaki (tcgen05 digit products, TMA tiles) + operand prep",
                "fp64_pipe_note": "the same update on native DFMA is FP64-pipe bound; see dfma_update"}
    elif wl.spec.k * (4 if wl.spec.kind == 1 else 1) <= 4:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": peak_hbm, "unit": "GB/s",
                "frac": achieved_gbs / peak_hbm, "traffic": None, "peak_kind": peak_kind,
                "kernel": "k_rank_update_c64_fp32 (rank <= 4, FP32 FMA stream on the CUDA cores)"}
    else:
        # 8 p flops per 16 bytes of G at p <= 128: far below the tensor pipe's flops per HBM byte
        f16_peak, f16_kind = f16_peak_tflops()
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": peak_hbm, "unit": "GB/s",
                "frac": achieved_gbs / peak_hbm, "traffic": None, "peak_kind": peak_kind,
                "kernel": "k_rank_update_c64_ra (p <= 48: resident A blocks) / k_rank_update_c64_wide (p > 48: "
                          "streaming 128 x 256 tiles); tcgen05 kind::f16, scaled split-FP16, 3 products; "
                          "+ D A^-1 + S GEMM + operand prep",
                "tensor_achieved_tflops": achieved_tfl, "tensor_peak_tflops": f16_peak, "tensor_peak_kind": f16_kind,
                "tensor_frac": achieved_tfl / f16_peak,
                "flops_note": "algorithmic 8 p n^2 per update (p rounded up to 16 executes); the split form runs 3 products"}
    roof["algorithmic_bytes_per_launch"] = bytes_per_launch
    roof["kernel_ms_avg"] = kern_avg_ms
    roof["kernel_share_of_step"] = kern_ms / ms
    # library kernels per step: eval, select (k = 1: one, two from 32768 candidates; top-k: begin
    # + k passes + end), capacitance, panels (not for complex64 on the tensor cores, which gathers
    # C0 with its row operands), finish, then per wavelength the update's launches and the bands
    pmax = wl.spec.k * (4 if wl.spec.kind == 1 else 1)
    sel = select_launches(ncand_main) if wl.spec.k <= 1 else wl.spec.k + 2
    if wl.dtype == "c128":
        upd = 3 if oz else 1                       # digit prep rows + cols + tensor-core update, or DFMA
    else:
        # FP32 stream, or inverse + S GEMM + C0 with the row operands + the resident-A update (+ the
        # streaming update where the workspace allows p > 48; it returns at once when p <= 48)
        upd = 1 if pmax <= 4 else (4 if pmax <= 48 else 5)
    panels = 0 if (wl.dtype == "c64" and pmax > 4) else 1
    # capacitance: the decision, after the per-wavelength solves of several wavelengths (p_max
    # <= 64) or the cluster solve of one wavelength's large set (64 < p_max <= 256)
    cap = 1 + (1 if (nlam > 1 and pmax <= 64) or (nlam == 1 and 64 < pmax <= 256) else 0)
    per_step_launches = 2 + sel + cap + panels + nlam * (upd + 1)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            # one GPU: the same problem the row-sharded runs split (strong scaling); replicas: weak
            "scaling": "weak" if world > 1 else "strong", "vs_baseline": None,
            "dtype": "f64" if wl.dtype == "c128" else "f32",
            "data": "synthetic",
            "config": {"workload": wl.name, "nx": g.nx, "ny": g.ny, "n": g.N + 1,
                       "candidates": ncand_main, "G_GB": G_GB_main,
                       "storage": wl.dtype, "k": wl.spec.k, "nlam": nlam,
                       "l2": "inputs larger than L2 (G is %.1f GB per replica)" % (G_GB_main * nlam),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "timed_as": "one CUDA-graph replay of the K steps" if args.graph else "K eager steps",
                       "update_algo": args.update_algo},
            "candidate_evals_per_s": ncand_main * args.steps * world / (t_max / 1e3),
            "g_update_GBps": achieved_gbs,
            "accepted_flips": flips_total,
            "roofline": roof,
            "gpu_launches": per_step_launches * args.steps,
            "clocks": clk,
            "e2e": e2e}
    if breakdown is not None:
        line["step_breakdown_ms"] = breakdown
    if args.graph and persistent_one is not None:
        line["persistent_batch_of_one"] = persistent_one
    if dfma is not None:
        line["dfma_update"] = dfma
    if refresh is not None:
        line["refresh"] = refresh
    if mixed is not None:
        line["mixed"] = mixed
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_budget, args.workload)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_egreedy(args):
    """Sec. V exploration study on the 21x21 metalens analogue: the greedy trajectory and
    20 seeded epsilon-greedy trajectories for each of epsilon = 0.1, 0.2, 0.3, every one run to
    termination, all 61 as problems of one fused batch (the persistent step kernel, one launch
    per step, 32 steps per CUDA graph replay).  Reported: accepted flips per second over the whole study
    (device-timed) and the final-FOM statistics per epsilon."""
    import torch
    from paper_2202_05388_gb300 import build as BLD
    from paper_2202_05388_gb300.egreedy import egreedy_study_batched

    torch.cuda.set_device(0)
    BLD.build()
    egreedy_study_batched(epsilons=(0.0, 0.1), trajectories=2, seed=99, max_steps=64)     # warm-up (kernel loading)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    res = egreedy_study_batched(epsilons=(0.0, 0.1, 0.2, 0.3), trajectories=20, seed=0, max_steps=4000)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    enq = res.pop("_steps_enqueued")
    flips = sum(r["steps_mean"] * r["trajectories"] for r in res.values())
    per_step = egreedy_step_forms()
    line = {"metric": METRIC + " [epsilon-greedy study, 61 trajectories batched]", "value": flips / (ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": int(enq), "warmup": 1, "ms_per_step": ms / max(enq, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "egreedy_21x21_single_c128", "trajectories_per_epsilon": 20, "problems": 61,
                       "schedule": "fused batch, 32-step CUDA graphs, run until every trajectory terminates",
                       "note": "ms_per_step is per batched step of all 61 trajectories"},
            "accepted_flips": int(round(flips)),
            "study": {str(e): {k: v for k, v in r.items() if k != "finals"} for e, r in res.items()},
            "batched_step_ms_by_form": per_step,
            "gpu_launches": int(enq) * 1, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def egreedy_step_forms(steps: int = 32):
    """Device time of one batched step of the study's 61 problems (a graph of `steps` steps from
    the filled start, replayed once after a warm-up replay from the same start), per fused form:
    the persistent launch with the FP64 FMA update (the default for these small problems, one
    launch per step), the same update in one launch per stage, and the persistent front launch
    with the tensor-core update (three launches per step)."""
    import torch
    from paper_2202_05388_gb300 import gfopt as B
    from paper_2202_05388_gb300.batch import BatchOptimizer, Schedule
    from paper_2202_05388_gb300.egreedy import metalens_21, _seed

    wl = metalens_21()
    pols = [None] + [(eps, _seed(0, e_i, t)) for e_i, eps in enumerate((0.1, 0.2, 0.3), start=1) for t in range(20)]
    out = {}
    for name, algo, form in (("persistent, FP64 FMA update (1 launch)", None, B.GF_BATCH_PERSISTENT),
                             ("staged, FP64 FMA update (7 launches)", None, B.GF_BATCH_STAGED),
                             ("persistent, tensor-core update (3 launches)", B.GF_UPDATE_TENSOR, B.GF_BATCH_PERSISTENT)):
        bo = BatchOptimizer([wl] * len(pols), dtype=wl.dtype, policies=pols, horizon=4 * steps + 8, update_algo=algo)
        bo.schedule = Schedule(0, "given", True, 0, form)
        times = []
        for _ in range(2):
            bo.fill()
            bo._policy_steps.zero_()
            bo.capture(steps)
            bo.fill()
            bo._policy_steps.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            bo.replay()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / steps)
        out[name] = min(times)
        bo.close()
        del bo
    return out


def run_deferred(args):
    """The 192x192 brush workload in the deferred (low-rank) form: no dense G; warm-up steps
    advance the run to a depth of W flips (the per-step cost grows with the stored columns K),
    then K steps are timed with CUDA events.  The dominant kernel is the column product
    (n x K by K x p, FP64)."""
    import torch
    from paper_2202_05388_gb300 import build as BLD
    from paper_2202_05388_gb300.deferred import DeferredOptimizer

    torch.cuda.set_device(0)
    BLD.build()
    wl = W.brush_192()
    g = wl.geoms[0]
    depth = max(3, args.warmup)
    opt = DeferredOptimizer(g, wl.spec, max_cols=4 * (depth + args.steps) + 8)
    opt.init()
    accepted = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(depth):
        opt.step()
        accepted += opt.applied.to(torch.int64)
    accepted.zero_()
    torch.cuda.synchronize()
    nt0, nc0 = opt.count()
    opt.h.gf_profile_begin(args.steps + 4)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        opt.step()
        accepted += opt.applied.to(torch.int64)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    kern_ms, kern_launches, _, flops = opt.h.gf_profile_end()
    nt1, nc1 = opt.count()
    flips = int(accepted.item())
    n = g.N + 1
    bytes_cols = 16.0 * n * args.steps * (nc0 + nc1) / 2.0        # U read once per step (K grows ~linearly)
    tflops = flops / (kern_ms * 1e-3) / 1e12 if kern_ms > 0 else 0.0
    fp64_peak = 152 * 2 * 2 * 2.07e9 / 1e12                        # nominal: 2 DFMA / SM / clk at 2.07 GHz
    peak_hbm, peak_kind = measured_peaks()
    line = {"metric": METRIC + " [deferred low-rank form]", "value": flips / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": depth, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "deferred_brush_192x192_p4", "n": n, "depth_flips_before_timing": nt0,
                       "stored_columns": [nc0, nc1], "U_GB": opt.U.numel() * 16 / 1e9,
                       "dense_G_GB": n * (n + (n & 1)) * 16 / 1e9,
                       "l2": "stored columns %.2f GB at the end; the column product reads them every step"
                             % (nc1 * n * 16 / 1e9)},
            "accepted_flips": flips,
            "roofline": {"bound": "alu", "achieved": tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": tflops / fp64_peak, "traffic": None,
                         "peak_kind": "nominal FP64 FMA rate (152 SMs x 2 DFMA/clk x 2.07 GHz)",
                         "kernel": "k_lr_columns (G0 column + n x K by K x p FP64 product)",
                         "kernel_ms_avg": kern_ms / max(kern_launches, 1),
                         "kernel_share_of_step": kern_ms / ms,
                         "hbm_achieved_gbs_approx": bytes_cols / (kern_ms * 1e-3) / 1e9 if kern_ms > 0 else 0.0,
                         "hbm_peak_gbs": peak_hbm},
            "gpu_launches": (6 + select_launches(opt.ncand)) * args.steps,
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_full(args, deferred: bool):
    """The whole greedy optimisation of the 192x192 brush workload, from the vacuum start to the
    design where no brush improves the FOM, timed end to end on the device (dense form: fill of
    the 21.7 GB G + every step; deferred form: init + every step).  The status word is read
    back every 32 steps; steps after termination are no-ops.  A warm-up run of a few steps
    loads every kernel first."""
    import torch
    from paper_2202_05388_gb300 import build as BLD
    from paper_2202_05388_gb300 import gfopt as B
    from paper_2202_05388_gb300.deferred import DeferredOptimizer
    from paper_2202_05388_gb300.optimizer import GreedyOptimizer

    torch.cuda.set_device(0)
    BLD.build()
    wl = W.brush_192()
    g = wl.geoms[0]
    max_steps = 4000

    def make():
        if deferred:
            o = DeferredOptimizer(g, wl.spec, max_cols=4 * max_steps + 8)
            return o, o.init
        o = GreedyOptimizer(wl.geoms, wl.spec)
        return o, o.fill

    opt, start = make()
    start()
    accepted = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(max(3, args.warmup)):          # the exact loop body, so every kernel is loaded
        opt.step()
        accepted += opt.applied.to(torch.int64)
    int(opt.status.cpu()[0])
    accepted.zero_()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    start()
    steps = 0
    marks = []
    while steps < max_steps:
        for _ in range(32):
            opt.step()
            accepted += opt.applied.to(torch.int64)
        steps += 32
        ev = torch.cuda.Event(enable_timing=True)
        ev.record()
        marks.append(ev)
        if int(opt.status.cpu()[0]) != B.GF_OK:
            break
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    flips = int(accepted.item())
    fom = float(opt.fom.cpu()[0])
    peak_hbm, peak_kind = measured_peaks()
    n = g.N + 1
    chunk_ms = [e0.elapsed_time(marks[0])] + [marks[i - 1].elapsed_time(marks[i]) for i in range(1, len(marks))]
    cfg = {"workload": ("deferred" if deferred else "dense") + "_brush_192x192_p4_to_termination", "n": n,
           "ms_per_32_steps": [round(x, 2) for x in chunk_ms],
           "flips_to_termination": flips, "final_fom": fom,
           "steps_enqueued": steps, "status_readback_every": 32,
           "memory_GB": (opt.U.numel() * 16 if deferred else opt.G[0].numel() * 16) / 1e9,
           "l2": "inputs larger than L2" if not deferred else "stored columns up to %.2f GB" % (4 * flips * n * 16 / 1e9)}
    line = {"metric": METRIC + " [whole optimisation to termination]", "value": flips / (ms / 1e3), "unit": UNIT,
            "n_gpus": 1, "steps": steps, "warmup": max(3, args.warmup), "ms_per_step": ms / max(flips, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg, "job_ms": ms, "accepted_flips": flips, "clocks": clk,
            "gpu_launches": steps * ((6 if deferred else 8) + select_launches(opt.ncand))}
    print(json.dumps(line), flush=True)
    return 0


def run_topk_run(args):
    """The 320x320 top-32 complex64 workload as a whole run: from the vacuum start for up to 1500
    steps (or until no brush improves the FOM), with the drift refresh every 200 steps: the field
    repair (GreedyOptimizer.refresh_fields: Eq. 3 residual of E, GMRES re-solve above 1e-5) and
    the Eq. 2 check of 8 sampled columns of G (gf_refresh).  Timed on the device from the fill to
    the last step, refreshes included; the refresh time is also reported per 200 steps."""
    import torch
    from paper_2202_05388_gb300 import build as BLD
    from paper_2202_05388_gb300 import gfopt as B
    from paper_2202_05388_gb300.optimizer import GreedyOptimizer

    torch.cuda.set_device(0)
    BLD.build()
    wl = W.brush_320_topk()
    g = wl.geoms[0]
    max_steps, every, chunk = 1500, 200, 25
    opt = GreedyOptimizer(wl.geoms, wl.spec, dtype=wl.dtype)
    opt.fill()
    for _ in range(3):                       # the exact loop body, so every kernel is loaded
        opt.step()
    opt.refresh_fields()
    opt.refresh(nsample=2)
    torch.cuda.synchronize()
    accepted = torch.zeros(1, dtype=torch.int64, device="cuda")
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall0 = time.perf_counter()
    e0.record()
    opt.fill()
    steps, refreshes = 0, []
    while steps < max_steps:
        for _ in range(chunk):
            opt.step()
            accepted += opt.applied.to(torch.int64)
        steps += chunk
        if int(opt.status.cpu()[0]) != B.GF_OK:
            break
        if steps % every == 0:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = opt.refresh_fields()[0]
            res, its, cres = opt.refresh(nsample=8)[0]
            torch.cuda.synchronize()
            refreshes.append({"step": steps, "seconds": time.perf_counter() - t0,
                              "e_residual": rep["e_residual"], "e_replaced": rep["e_replaced"],
                              "e_residual_after": rep["e_residual_after"], "e_gmres_iters": rep["e_iters"],
                              "ls_residual": res[0], "column_residual_max": max(cres), "column_gmres_iters": its})
    e1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    flips = int(accepted.item())
    t_ref = sum(r["seconds"] for r in refreshes)
    # the drift check of the final design (outside the timed region): the run may end before its
    # first scheduled refresh, and this one certifies the state the run returns
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = opt.refresh_fields()[0]
    res, its, cres = opt.refresh(nsample=8)[0]
    torch.cuda.synchronize()
    final_check = {"step": steps, "seconds": time.perf_counter() - t0, "e_residual": rep["e_residual"],
                   "e_replaced": rep["e_replaced"], "e_residual_after": rep["e_residual_after"],
                   "e_gmres_iters": rep["e_iters"], "ls_residual": res[0], "column_residual_max": max(cres),
                   "column_gmres_iters": its}
    per_refresh = [r["seconds"] for r in refreshes] + [final_check["seconds"]]
    refresh_s = sum(per_refresh) / len(per_refresh)
    line = {"metric": METRIC + " [320x320 top-32 whole run with drift refresh]", "value": flips / (ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": 3, "ms_per_step": ms / max(steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name + "_run_refresh200", "n": g.N + 1, "max_steps": max_steps,
                       "refresh_every": every, "status_readback_every": chunk, "l2": "inputs larger than L2"},
            "job_s": ms / 1e3, "wall_s": wall, "accepted_flips": flips, "final_fom": float(opt.fom.cpu()[0]),
            "refresh": {"count_in_run": len(refreshes), "seconds_in_run": t_ref,
                        "seconds_per_refresh": refresh_s,
                        # one refresh per 200 steps: its cost against 200 steps at this run's rate
                        "overhead_per_200_steps_s": refresh_s,
                        "overhead_share_at_every_200": refresh_s / (refresh_s + 200 * ms / max(steps, 1) / 1e3),
                        "records": refreshes, "final_check": final_check},
            # per step: dFOM 1, top-32 selection 34 (begin, 32 passes, end), capacitance 2 (the
            # cluster solve, the decision), complex64 update 5 (D A^-1, S GEMM, C0 with the row
            # operands, both forms), field/FOM 1, bands 1
            "gpu_launches": 44 * steps, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_metalens3d(args):
    """Sec. IV's metalens in its own 3-D form: 120 x 120 x 4 voxels of lambda/20 (75 nm at
    lambda = 1.5 um), silicon pillars (2x2 lateral, all 4 layers: 48 unknowns per flip), x-polarised
    plane wave, focus 3 lambda past the slab (NA 0.7), dyadic G over 172 803 unknowns in complex64
    (239 GB).  Every one of the 28 322 pillar candidates (both directions, all anchors) is
    evaluated each step; the accepted flip is applied as a rank-48 update on the tensor cores."""
    import torch
    from paper_2202_05388_gb300 import build as BLD
    from paper_2202_05388_gb300 import gfopt as B
    from paper_2202_05388_gb300.optimizer import GreedyOptimizer3D

    torch.cuda.set_device(0)
    BLD.build()
    wl = W.metalens_3d(nx=32, ny=32) if args.workload == "metalens3d_32" else W.metalens_3d()
    g = wl.geoms[0]
    opt = GreedyOptimizer3D(g, wl.spec, dtype="c64")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    opt.fill()
    torch.cuda.synchronize()
    e0.record()
    opt.fill()
    e1.record()
    torch.cuda.synchronize()
    fill_ms = e0.elapsed_time(e1)
    accepted = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(max(3, args.warmup)):
        opt.step()
        accepted += opt.applied.to(torch.int64)
    int(opt.status.cpu()[0])
    accepted.zero_()
    torch.cuda.synchronize()
    opt.h.gf_profile_begin(args.steps + 4)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    e0.record()
    for _ in range(args.steps):
        opt.step()
        accepted += opt.applied.to(torch.int64)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    kern_ms, kern_n, kern_bytes, kern_flops = opt.h.gf_profile_end()
    flips = int(accepted.item())
    # stage breakdown over two more steps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    br = {"eval": 0.0, "select": 0.0, "update": 0.0}
    for _ in range(2):
        ev[0].record()
        opt.evaluate()
        ev[1].record()
        opt.select()
        ev[2].record()
        opt.update()
        ev[3].record()
        torch.cuda.synchronize()
        br["eval"] += ev[0].elapsed_time(ev[1]) / 2
        br["select"] += ev[1].elapsed_time(ev[2]) / 2
        br["update"] += ev[2].elapsed_time(ev[3]) / 2
    peak_hbm, peak_kind = measured_peaks()
    kavg = kern_ms / max(kern_n, 1)
    bpl = kern_bytes / max(kern_n, 1)
    gbs = bpl / (kavg * 1e-3) / 1e9 if kavg > 0 else 0.0
    paper_step_s = 3.7 * 60.0
    line = {"metric": METRIC.replace("2x2 brush", "2x2x4 pillar") + " [3-D metalens]", "value": flips / (ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": (flips / (ms / 1e3)) / (1.0 / paper_step_s),
            "vs_baseline_note": "the paper's run of this metalens: 3.7 min per step (one accepted flip per step) on "
                                "2000 CPU workers with 3600 aligned 2x2 candidates; here every one of the 28322 "
                                "pillar positions is evaluated each step",
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "voxels": [g.nx, g.ny, g.nz], "unknowns": opt.n,
                       "candidates": opt.ncand, "G_GB": opt.G.numel() * 8 / 1e9, "storage": "c64",
                       "l2": "inputs larger than L2 (G is %.0f GB)" % (opt.G.numel() * 8 / 1e9)},
            "accepted_flips": flips, "fill_ms": fill_ms, "step_breakdown_ms": br,
            "candidate_evals_per_s": opt.ncand * args.steps / (ms / 1e3),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak_hbm, "unit": "GB/s", "frac": gbs / peak_hbm,
                         "traffic": None, "peak_kind": peak_kind,
                         "kernel": "k_rank_update_c64_ra (rank 3p, split-FP16 tensor cores, resident A blocks)",
                         "kernel_ms_avg": kavg, "algorithmic_bytes_per_launch": bpl,
                         "tflops_achieved": kern_flops / max(kern_n, 1) / (kavg * 1e-3) / 1e12 if kavg > 0 else 0.0},
            "gpu_launches": 9 * args.steps, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_metalens3d_full(args):
    """The whole greedy optimisation of the 3-D metalens, from the vacuum slab until no pillar
    improves the focal intensity (the paper's run took 750 steps of 3.7 min), timed end to end
    on the device: fill + every step (status read back every 25 steps)."""
    import torch
    from paper_2202_05388_gb300 import build as BLD
    from paper_2202_05388_gb300 import gfopt as B
    from paper_2202_05388_gb300.optimizer import GreedyOptimizer3D

    torch.cuda.set_device(0)
    BLD.build()
    wl = (W.metalens_3d_aligned(fill_only="fill" in args.workload) if "aligned" in args.workload
          else W.metalens_3d())
    g = wl.geoms[0]
    opt = GreedyOptimizer3D(g, wl.spec, dtype="c64")
    accepted = torch.zeros(1, dtype=torch.int64, device="cuda")
    opt.fill()
    for _ in range(3):                                  # warm-up: the exact loop body
        opt.step()
        accepted += opt.applied.to(torch.int64)
    int(opt.status.cpu()[0])
    accepted.zero_()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    opt.fill()
    fom0 = float(opt.fom.cpu()[0])
    steps = 0
    trace = []
    while steps < 4000:
        for _ in range(25):
            opt.step()
            accepted += opt.applied.to(torch.int64)
        steps += 25
        st, fom = int(opt.status.cpu()[0]), float(opt.fom.cpu()[0])
        trace.append(round(fom / fom0, 4))
        if st != B.GF_OK:
            break
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    flips = int(accepted.item())
    line = {"metric": METRIC.replace("2x2 brush", "2x2x4 pillar") + " [3-D metalens, whole optimisation]",
            "value": flips / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": 3,
            "ms_per_step": ms / max(flips, 1), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name + "_to_termination", "voxels": [g.nx, g.ny, g.nz], "unknowns": opt.n,
                       "status_readback_every": 25, "l2": "inputs larger than L2"},
            "job_s": ms / 1e3, "accepted_flips": flips, "final_fom_over_initial": trace[-1] if trace else 1.0,
            "fom_over_initial_every_25_steps": trace,
            "paper_context": "the paper's run of this lens: 750 steps of 3.7 min (about 46 h) on 2000 CPU workers",
            "gpu_launches": 9 * steps, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.oracle_sample:
        name, budget = args.oracle_sample.split(":")
        step, desc, parts = oracle_step_sample(workload(name), float(budget))
        print(json.dumps({"seconds_per_step": step, "parts_s": parts, "sample": desc}), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    if args.workload.startswith("batch_48"):
        return run_batch(args)
    if args.workload == "egreedy_21x21":
        return run_egreedy(args)
    if args.workload == "deferred_192":
        return run_deferred(args)
    if args.workload in ("metalens3d", "metalens3d_32"):
        return run_metalens3d(args)
    if args.workload in ("metalens3d_run", "metalens3d_aligned_run", "metalens3d_aligned_fill_run"):
        return run_metalens3d_full(args)
    if args.workload == "brush_320_topk_run":
        return run_topk_run(args)
    if args.workload in ("deferred_192_run", "brush_192_run"):
        return run_full(args, deferred=args.workload.startswith("deferred"))
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
