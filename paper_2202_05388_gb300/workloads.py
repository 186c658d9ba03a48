"""Synthetic workload recipes (inputs only; none of the method's arithmetic).

Every workload is a 2-D scalar (E_z) restatement of the paper's metalens problem
(Sec. IV): a rectangular design grid of nx*ny square pixels of side dx in a vacuum
background, binary permittivity {eps_bg, eps_mat}, a plane wave travelling +y and one
monitor (focal) point outside the design region on its centre line.  These records are
shared by the CUDA path, the tests, the bench and the oracle; they hold numbers only.

Geometry conventions (shared input convention, not arithmetic of the method):
  * pixel j = iy*nx + ix, centre ((ix+1/2)dx, (iy+1/2)dx); the design region spans
    x in [0, nx*dx], y in [0, ny*dx];
  * the monitor point is index N = nx*ny of every Green's matrix (n = N+1 points);
  * the design starts at eps_bg everywhere (state 0).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass
from typing import List

import numpy as np

KIND_SINGLE = 0     # one pixel per candidate, id = j
KIND_BRUSH2 = 1     # 2x2 brush per candidate, id = dir*P + iy*(nx-1) + ix
KIND_PILLAR = 2     # 3-D: 2x2 lateral block through all nz layers, id as for KIND_BRUSH2
DIR_FILL = 1        # eps_bg -> eps_mat
DIR_CLEAR = 2       # eps_mat -> eps_bg


@dataclass(frozen=True)
class Geometry:
    nx: int
    ny: int
    dx: float
    wavelength: float
    mon_x: float
    mon_y: float
    eps_bg: float = 1.0
    eps_mat: float = 12.25

    @property
    def N(self) -> int:
        return self.nx * self.ny

    @property
    def n(self) -> int:
        return self.nx * self.ny + 1


@dataclass(frozen=True)
class Geometry3D:
    """3-D slab of nx*ny*nz cubic voxels of side dx (Sec. IV's metalens: a slab in the xy plane,
    thickness along z); plane wave polarised along x travelling +z; one monitor point.
    Voxel j = (iz*ny + iy)*nx + ix, centre ((ix+1/2)dx, (iy+1/2)dx, (iz+1/2)dx); the monitor is
    point N; unknown u = 3*point + component (x, y, z)."""
    nx: int
    ny: int
    nz: int
    dx: float
    wavelength: float
    mon_x: float
    mon_y: float
    mon_z: float
    eps_bg: float = 1.0
    eps_mat: float = 12.0

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n(self) -> int:
        return 3 * (self.N + 1)


@dataclass(frozen=True)
class CandidateSpec:
    kind: int = KIND_SINGLE
    dir_mask: int = DIR_FILL
    k: int = 1                 # flips accepted per step (top-k with exclusion when k > 1)
    excl_radius: int = 3       # Chebyshev distance between anchors that counts as a conflict
    tie_rel: float = 1e-12     # relative window of the lowest-index tie rule
    aligned: bool = False      # brushes / pillars: only even anchors (Sec. IV's aligned 2x2 partitions)

    def ncand(self, g) -> int:
        if self.kind == KIND_SINGLE:
            return g.N
        return 2 * (g.nx - 1) * (g.ny - 1)


@dataclass(frozen=True)
class Workload:
    name: str
    geoms: tuple            # one Geometry per wavelength (multi-wavelength FOM sums over them)
    spec: CandidateSpec
    steps: int
    dtype: str              # "c128" or "c64"


def _centre_line_monitor(nx, ny, dx, beyond_centre=None, beyond_edge=None):
    x = nx * dx / 2.0
    if beyond_centre is not None:
        return x, ny * dx / 2.0 + beyond_centre
    return x, ny * dx + beyond_edge


def plain_32() -> Workload:
    """32x32 pixels, lambda = 1, dx = lambda/20, single-pixel fill flips, 100 steps;
    monitor 2 lambda past the far edge on the centre line."""
    nx = ny = 32
    dx = 0.05
    mx, my = _centre_line_monitor(nx, ny, dx, beyond_edge=2.0)
    g = Geometry(nx, ny, dx, 1.0, mx, my)
    return Workload("plain_32x32_single_c128", (g,), CandidateSpec(KIND_SINGLE, DIR_FILL, 1),
                    100, "c128")


def brush_192() -> Workload:
    """192x192 pixels, dx = lambda/20, every 2x2 brush toggle in both directions,
    focus 5 lambda beyond the region centre, complex128 G (about 21.7 GB), 2000 steps."""
    nx = ny = 192
    dx = 0.05
    mx, my = _centre_line_monitor(nx, ny, dx, beyond_centre=5.0)
    g = Geometry(nx, ny, dx, 1.0, mx, my)
    return Workload("brush_192x192_p4_c128", (g,),
                    CandidateSpec(KIND_BRUSH2, DIR_FILL | DIR_CLEAR, 1), 2000, "c128")


def brush_64() -> Workload:
    """64x64 pixels, dx = lambda/20, 2x2 brush toggles, focus 2 lambda beyond the centre:
    a profiling-size member of the brush family (G = 269 MB, larger than L2)."""
    nx = ny = 64
    dx = 0.05
    mx, my = _centre_line_monitor(nx, ny, dx, beyond_centre=2.0)
    g = Geometry(nx, ny, dx, 1.0, mx, my)
    return Workload("brush_64x64_p4_c128", (g,),
                    CandidateSpec(KIND_BRUSH2, DIR_FILL | DIR_CLEAR, 1), 200, "c128")


def brush_128() -> Workload:
    """128x128 member of the complex128 brush family (G = 4.3 GB): a capture-size case for the
    DRAM counters of the update (larger than L2 by 33x, a few GB on the device)."""
    nx = ny = 128
    dx = 0.05
    mx, my = _centre_line_monitor(nx, ny, dx, beyond_centre=5.0)
    g = Geometry(nx, ny, dx, 1.0, mx, my)
    return Workload("brush_128x128_p4_c128", (g,),
                    CandidateSpec(KIND_BRUSH2, DIR_FILL | DIR_CLEAR, 1), 200, "c128")


def brush_320_topk() -> Workload:
    """320x320 pixels, complex64 G (about 84 GB), top-32 brushes with a 3-pixel
    exclusion radius accepted per step as one rank-128 update, 1500 steps.  The focus is 5
    lambda past the far edge (NA 0.85): 5 lambda beyond the centre would lie inside this
    16-lambda-tall region."""
    nx = ny = 320
    dx = 0.05
    mx, my = _centre_line_monitor(nx, ny, dx, beyond_edge=5.0)
    g = Geometry(nx, ny, dx, 1.0, mx, my)
    return Workload("brush_320x320_top32_c64", (g,),
                    CandidateSpec(KIND_BRUSH2, DIR_FILL | DIR_CLEAR, 32, 3), 1500, "c64")


def brush_320_c128() -> Workload:
    """The 320x320 geometry of brush_320_topk with the plain FP64 form: complex128 G
    (168 GB), one brush (rank 4) per step -- the comparison point for the mixed form."""
    w = brush_320_topk()
    return Workload("brush_320x320_p4_c128", w.geoms, CandidateSpec(KIND_BRUSH2, DIR_FILL | DIR_CLEAR, 1),
                    w.steps, "c128")


def brush_320_c64_rank4() -> Workload:
    """The 320x320 geometry with complex64 G and one brush (rank 4) per step: the rank-4
    baseline form of the mixed-precision family."""
    w = brush_320_topk()
    return Workload("brush_320x320_p4_c64", w.geoms, CandidateSpec(KIND_BRUSH2, DIR_FILL | DIR_CLEAR, 1),
                    w.steps, "c64")


def brush_96_c64_rank4() -> Workload:
    """96x96 member of the complex64 rank-4 family (G = 680 MB, larger than L2), for profiling."""
    nx = ny = 96
    dx = 0.05
    mx, my = _centre_line_monitor(nx, ny, dx, beyond_edge=5.0)
    g = Geometry(nx, ny, dx, 1.0, mx, my)
    return Workload("brush_96x96_p4_c64", (g,), CandidateSpec(KIND_BRUSH2, DIR_FILL | DIR_CLEAR, 1), 200, "c64")


def brush_128_topk() -> Workload:
    """128x128 member of the top-32 complex64 family (G = 2.1 GB), for profiling."""
    nx = ny = 128
    dx = 0.05
    mx, my = _centre_line_monitor(nx, ny, dx, beyond_edge=5.0)
    g = Geometry(nx, ny, dx, 1.0, mx, my)
    return Workload("brush_128x128_top32_c64", (g,),
                    CandidateSpec(KIND_BRUSH2, DIR_FILL | DIR_CLEAR, 32, 3), 200, "c64")


def multi_lambda_512x64() -> Workload:
    """512x64 pixels, dx = lambda0/20, lambda in {0.9, 1.0, 1.1} lambda0, shared focus
    8 lambda0 beyond the region centre, FOM summed over wavelengths, top-16 brushes."""
    nx, ny = 512, 64
    dx = 0.05
    mx, my = _centre_line_monitor(nx, ny, dx, beyond_centre=8.0)
    geoms = tuple(Geometry(nx, ny, dx, lam, mx, my) for lam in (0.9, 1.0, 1.1))
    return Workload("multilambda_512x64_top16_c64", geoms,
                    CandidateSpec(KIND_BRUSH2, DIR_FILL | DIR_CLEAR, 16, 3), 1000, "c64")


def batch_48(seed: int = 2202, count: int = 48) -> List[Workload]:
    """48 independent problems: square side from {32,48,64,96,128}, lambda/dx from
    {16,20,24}, focus 2-6 lambda past the far edge, single-pixel toggles, 500 steps."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        side = int(rng.choice([32, 48, 64, 96, 128]))
        ratio = int(rng.choice([16, 20, 24]))
        focus = float(rng.uniform(2.0, 6.0))
        dx = 1.0 / ratio
        mx, my = _centre_line_monitor(side, side, dx, beyond_edge=focus)
        g = Geometry(side, side, dx, 1.0, mx, my)
        out.append(Workload(f"batch{b}_{side}x{side}_r{ratio}", (g,),
                            CandidateSpec(KIND_SINGLE, DIR_FILL | DIR_CLEAR, 1), 500, "c128"))
    return out


def small(nx: int, ny: int, kind: int = KIND_SINGLE, dir_mask: int = DIR_FILL, k: int = 1,
          excl_radius: int = 3, ratio: int = 20, beyond_edge: float = 2.0,
          wavelengths=(1.0,), steps: int = 10, dtype: str = "c128") -> Workload:
    """A small grid of the same shape family, for parity tests."""
    dx = 1.0 / ratio
    mx, my = _centre_line_monitor(nx, ny, dx, beyond_edge=beyond_edge)
    geoms = tuple(Geometry(nx, ny, dx, lam, mx, my) for lam in wavelengths)
    return Workload(f"small_{nx}x{ny}_k{kind}", geoms,
                    CandidateSpec(kind, dir_mask, k, excl_radius), steps, dtype)


def with_monitor(g: Geometry, mon_x: float, mon_y: float) -> Geometry:
    return dataclasses.replace(g, mon_x=mon_x, mon_y=mon_y)


def random_state(N: int, seed: int, fill: float = 0.3) -> np.ndarray:
    """Seeded random binary design (uint8), for tests that start from a patterned design."""
    rng = np.random.default_rng(seed)
    return (rng.random(N) < fill).astype(np.uint8)


def metalens_3d(nx: int = 120, ny: int = 120, nz: int = 4, na: float = 0.7, eps_mat: float = 12.0,
                dtype: str = "c64") -> Workload:
    """Sec. IV's metalens: nx x ny x nz voxels of lambda/20 (75 nm at lambda = 1.5 um: a
    9 um x 9 um x 300 nm silicon slab for 120 x 120 x 4), x-polarised plane wave at normal
    incidence, focus on the axis past the slab at the distance giving numerical aperture `na`
    (4.5 um = 3 lambda for NA 0.7), pillar (2x2 x nz) flips in both directions."""
    dx = 0.05
    half = nx * dx / 2.0
    import math
    f = half / math.tan(math.asin(na))
    g = Geometry3D(nx, ny, nz, dx, 1.0, half, ny * dx / 2.0, nz * dx + f, eps_mat=eps_mat)
    return Workload(f"metalens3d_{nx}x{ny}x{nz}_pillar_{dtype}", (g,),
                    CandidateSpec(KIND_PILLAR, DIR_FILL | DIR_CLEAR, 1), 750, dtype)


def metalens_3d_aligned(fill_only: bool = False) -> Workload:
    """metalens_3d with the paper's candidate set: the 60 x 60 aligned 2x2 partitions (and, with
    fill_only, blocks of silicon added to the vacuum slab only)."""
    w = metalens_3d()
    tag = "aligned_fill_pillar" if fill_only else "aligned_pillar"
    return Workload(w.name.replace("pillar", tag), w.geoms,
                    CandidateSpec(KIND_PILLAR, DIR_FILL if fill_only else DIR_FILL | DIR_CLEAR, 1, aligned=True),
                    w.steps, w.dtype)


def small_3d(nx: int, ny: int, nz: int, focus: float = 1.0, eps_mat: float = 12.0, k: int = 1,
             dtype: str = "c128") -> Workload:
    """A small 3-D slab of the same family, for parity tests."""
    dx = 0.05
    g = Geometry3D(nx, ny, nz, dx, 1.0, nx * dx / 2.0, ny * dx / 2.0, nz * dx + focus, eps_mat=eps_mat)
    return Workload(f"small3d_{nx}x{ny}x{nz}", (g,), CandidateSpec(KIND_PILLAR, DIR_FILL | DIR_CLEAR, k), 10, dtype)
