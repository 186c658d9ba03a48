"""The synthetic workloads against the values the paper prints for its own (Sec. IV metalens,
Sec. V exploration study; tests/golden/paper_workloads.json holds each value with its section).

Lengths are in units of the wavelength in the library, so 1 unit = 1500 nm here."""
import inspect
import json
import math
import os

import numpy as np

from oracle import gf_oracle3d as O3
from paper_2202_05388_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "paper_workloads.json")) as fh:
    GOLD = json.load(fh)
LENS = {k: v["value"] for k, v in GOLD["metalens"].items()}
STUDY = {k: v["value"] for k, v in GOLD["egreedy"].items()}
NM = LENS["wavelength_nm"]                      # nm per length unit


def _complex64_bytes(n: int) -> int:
    return 8 * n * n


def test_metalens_geometry_is_the_papers():
    g = W.metalens_3d().geoms[0]
    assert g.wavelength == 1.0
    assert [g.nx, g.ny] == LENS["lateral_pixels"]
    assert math.isclose(g.nx * g.dx * NM, LENS["side_um"] * 1e3)
    assert math.isclose(g.nz * g.dx * NM, LENS["thickness_nm"])
    assert g.eps_bg == LENS["eps_background"] and g.eps_mat == LENS["eps_pattern"]
    assert math.isclose(2 * g.dx * NM, LENS["min_feature_nm"])      # a 2 x 2 partition spans 150 nm
    # focus on the axis past the slab's top face: NA from the half aperture and that distance
    half = g.nx * g.dx / 2.0
    assert math.isclose(g.mon_x, half) and math.isclose(g.mon_y, g.ny * g.dx / 2.0)
    f = g.mon_z - g.nz * g.dx
    assert math.isclose(half / math.hypot(half, f), LENS["numerical_aperture"], rel_tol=1e-12)
    # the paper's two figures (4.5 um and NA 0.7) agree to 2%: sin(atan(4.5 / 4.5)) = 0.707
    assert abs(f * NM / 1e3 - LENS["focal_distance_um"]) / LENS["focal_distance_um"] < 0.03


def test_aligned_candidate_set_is_the_papers_partitions():
    w = W.metalens_3d_aligned(fill_only=True)
    g, spec = w.geoms[0], w.spec
    state = np.zeros(g.nx * g.ny * g.nz, dtype=np.uint8)
    live = [cid for cid in range(O3.num_candidates(g, spec)) if O3.candidate(g, spec, state, cid)[0].size]
    assert len(live) == LENS["partitions"]
    px, py = LENS["partition_pixels"]
    V, _ = O3.candidate(g, spec, state, live[0])
    assert V.size == 3 * px * py * g.nz                     # three field components per voxel
    # the partitions tile the lateral region without overlap
    covered = set()
    for cid in live:
        vox = set((O3.candidate(g, spec, state, cid)[0] // 3).tolist())
        assert not covered & vox
        covered |= vox
    assert len(covered) == g.nx * g.ny * g.nz


def test_green_matrix_size_matches_the_papers_inputs_per_step():
    """The partitions' inputs are G's row chunks (plus O(N) field and monitor terms), so their
    sum is G's size: the complex64 dyadic G of the 120 x 120 x 4 lens is 222.5 GiB against the
    printed 220 GiB.  At 50 nm per pixel the same slab has 180 x 180 x 6 voxels, and G grows by
    (1.5^3)^2 to 2.45 TiB; the paper's "about 2 TiB" is read as within 30%."""
    g = W.metalens_3d().geoms[0]
    n = g.n
    assert n == 3 * (g.nx * g.ny * g.nz + 1)
    gib = _complex64_bytes(n) / 2 ** 30
    assert abs(gib - LENS["inputs_per_step_GiB"]) / LENS["inputs_per_step_GiB"] < 0.02
    nx50 = round(LENS["side_um"] * 1e3 / 50)
    nz50 = round(LENS["thickness_nm"] / 50)
    g50 = W.metalens_3d(nx=nx50, ny=nx50, nz=nz50).geoms[0]
    tib = _complex64_bytes(g50.n) / 2 ** 40
    assert abs(tib - LENS["inputs_per_step_at_50nm_TiB"]) / LENS["inputs_per_step_at_50nm_TiB"] < 0.3
    assert math.isclose(tib * 1024 / gib, (g50.n / n) ** 2)


def test_exploration_study_geometry_and_protocol():
    from paper_2202_05388_gb300 import egreedy as EG
    g = EG.metalens_21().geoms[0]
    assert [g.nx, g.ny] == STUDY["pixels"]
    assert math.isclose(g.dx * NM, STUDY["pixel_nm"])
    half = g.nx * g.dx / 2.0
    f = g.mon_y - g.ny * g.dx                           # past the far edge, on the centre line
    assert math.isclose(g.mon_x, half)
    assert math.isclose(half / math.hypot(half, f), STUDY["numerical_aperture"], rel_tol=1e-12)
    sig = inspect.signature(EG.egreedy_study)
    eps = sig.parameters["epsilons"].default
    assert 0.0 in eps and sorted(e for e in eps if e > 0) == STUDY["epsilons"]
    assert sig.parameters["trajectories"].default == STUDY["runs_per_epsilon"]
