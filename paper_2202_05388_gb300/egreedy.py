"""The exploration study of Sec. V on a 2-D analogue: a 21x21-pixel focusing metalens
(dx = lambda/20, focus on the centre line at NA 0.7 past the far edge) optimised to
termination by the greedy policy and by epsilon-greedy policies, many seeded trajectories
per epsilon.  Every step runs in libgfopt through GreedyOptimizer; this module only drives
trajectories and summarises their final FOM.
"""
from __future__ import annotations

import math
from typing import Optional, Dict, List, Sequence

import numpy as np

import torch

from . import gfopt as B
from .batch import BatchOptimizer
from .optimizer import GreedyOptimizer
from .workloads import CandidateSpec, Geometry, KIND_SINGLE, DIR_FILL, DIR_CLEAR, Workload


def metalens_21(na: float = 0.7, eps_mat: float = 12.0) -> Workload:
    """21x21 pixels of lambda/20 (the 75 nm pixels of Sec. V at lambda = 1.5 um), silicon
    pixels, single-pixel toggles, focus on the centre line at the distance past the far edge
    that gives the numerical aperture `na` for the lens aperture."""
    n = 21
    dx = 0.05
    half = n * dx / 2.0
    f = half / math.tan(math.asin(na))
    g = Geometry(n, n, dx, 1.0, half, n * dx + f, eps_mat=eps_mat)
    return Workload("metalens_21x21_single", (g,), CandidateSpec(KIND_SINGLE, DIR_FILL | DIR_CLEAR, 1), 2000, "c128")


def run_to_termination(opt: GreedyOptimizer, max_steps: int) -> List[float]:
    """FOM after every step until no improving action is left (or max_steps)."""
    trace = []
    for _ in range(max_steps):
        opt.step()
        r = opt.read_step()
        if r.status != B.GF_OK:
            break
        trace.append(r.fom)
    return trace


def egreedy_study(epsilons: Sequence[float] = (0.0, 0.1, 0.2, 0.3), trajectories: int = 20, seed: int = 0,
                  max_steps: int = 4000, device: int = 0, update_algo: Optional[int] = None) -> Dict[float, dict]:
    """Final-FOM statistics per epsilon over seeded trajectories (epsilon = 0 is the greedy
    policy; its trajectories are all the same).  update_algo: the G update's arithmetic
    (gf_set_update_algo; the library default when None, which for these small problems is the
    FP64 FMA form -- the fused batch's arithmetic exactly)."""
    wl = metalens_21()
    out = {}
    for e_i, eps in enumerate(epsilons):
        finals, steps = [], []
        for t in range(trajectories if eps > 0 else 1):
            opt = GreedyOptimizer(wl.geoms, wl.spec, dtype=wl.dtype, device=device)
            if update_algo is not None:
                opt.h.gf_set_update_algo(update_algo)
            opt.fill()
            fom0 = float(opt.fom.cpu()[0])
            if eps > 0:
                opt.set_egreedy(eps, seed=_seed(seed, e_i, t), horizon=max_steps + 1)
            trace = run_to_termination(opt, max_steps)
            finals.append((trace[-1] if trace else fom0) / fom0)
            steps.append(len(trace))
        f = np.array(finals)
        out[eps] = {"trajectories": len(finals), "final_fom_mean": float(f.mean()), "final_fom_std": float(f.std()),
                    "final_fom_max": float(f.max()), "final_fom_min": float(f.min()),
                    "steps_mean": float(np.mean(steps)), "finals": finals}
    return out


def _seed(seed: int, e_i: int, t: int) -> int:
    return seed * 1000003 + e_i * 1009 + t


def egreedy_study_batched(epsilons: Sequence[float] = (0.0, 0.1, 0.2, 0.3), trajectories: int = 20,
                          seed: int = 0, max_steps: int = 4000, device: int = 0, chunk: int = 32) -> Dict[float, dict]:
    """The same study with every trajectory a problem of one fused batch (the persistent step
    kernel: one launch per step of all of them, chunk steps per CUDA graph), run until every
    trajectory has no improving action left.  Same seeds as egreedy_study, so the same
    trajectories."""
    wl = metalens_21()
    pols, owner = [], []
    for e_i, eps in enumerate(epsilons):
        for t in range(trajectories if eps > 0 else 1):
            pols.append((eps, _seed(seed, e_i, t)) if eps > 0 else None)
            owner.append(eps)
    bo = BatchOptimizer([wl] * len(pols), dtype=wl.dtype, device=device, policies=pols, horizon=max_steps + 2 * chunk)
    bo.fill()
    fom0 = float(bo.opts[0].fom.cpu()[0])
    bo.capture(chunk)                       # one step runs before the capture
    steps = 1
    while steps < max_steps:
        bo.replay()
        steps += chunk
        status = torch.stack([o.status for o in bo.opts]).cpu().numpy().ravel()
        if (status != B.GF_OK).all():
            break
    applied = bo.applied.cpu().numpy()
    foms = [float(o.fom.cpu()[0]) / fom0 for o in bo.opts]
    out = {}
    for eps in epsilons:
        sel = [i for i, e in enumerate(owner) if e == eps]
        f = np.array([foms[i] for i in sel])
        out[eps] = {"trajectories": len(sel), "final_fom_mean": float(f.mean()), "final_fom_std": float(f.std()),
                    "final_fom_max": float(f.max()), "final_fom_min": float(f.min()),
                    "steps_mean": float(np.mean([applied[i] for i in sel])), "finals": [foms[i] for i in sel]}
    out["_steps_enqueued"] = steps
    bo.close()
    return out
