"""The arithmetic of the 3-D pillar evaluation for complex64 G (each candidate's system factorised
in FP32 with partial pivoting -- largest |a|^2, lowest row on ties -- and the solution refined
once with the residual b - A y formed in FP64 from the stored entries), restated in numpy and
run on the pillar systems of the 3-D oracle's matrices: the refined solution is the FP64 solve
of the same stored system to ~1e-12, the unrefined FP32 one is not, and the first correction
stays far below the 2^-10 singularity flag."""
import numpy as np
import pytest

from oracle import gf_oracle as O
from oracle import gf_oracle3d as O3
from paper_2202_05388_gb300 import workloads as W


def _lu32(A):
    """FP32 LU with partial pivoting (row interchanges applied to whole rows)."""
    A = A.astype(np.complex64).copy()
    p = A.shape[0]
    piv = np.arange(p)
    for c in range(p):
        mag = (A[c:, c].real.astype(np.float32) ** 2 + A[c:, c].imag.astype(np.float32) ** 2)
        r = c + int(np.argmax(mag))                    # first maximum: the lowest row on ties
        if r != c:
            A[[c, r]] = A[[r, c]]
            piv[[c, r]] = piv[[r, c]]
        A[c + 1:, c] = A[c + 1:, c] * (np.complex64(1) / A[c, c])
        A[c + 1:, c + 1:] -= np.outer(A[c + 1:, c], A[c, c + 1:]).astype(np.complex64)
    return A, piv


def _solve32(LU, piv, b):
    y = b.astype(np.complex64)[piv].copy()
    p = len(y)
    for r in range(1, p):
        y[r] -= np.dot(LU[r, :r], y[:r])
    for r in range(p - 1, -1, -1):
        y[r] = (y[r] - np.dot(LU[r, r + 1:], y[r + 1:])) / LU[r, r]
    return y


@pytest.mark.parametrize("nx,ny,nz,fill,seed", [(6, 6, 2, 0.3, 1), (5, 5, 4, 0.4, 2)])
def test_fp32_factors_with_one_fp64_refinement_reach_the_fp64_solve(nx, ny, nz, fill, seed):
    g = W.small_3d(nx, ny, nz).geoms[0]
    spec = W.CandidateSpec(W.KIND_PILLAR, 3, 1)
    state = (np.random.default_rng(seed).random(nx * ny * nz) < fill).astype(np.uint8)
    G, E = O3.brute_force(g, state)
    Gs = G.astype(np.complex64).astype(np.complex128)  # the stored complex64 matrix
    worst_ir = worst_plain = worst_corr = 0.0
    count = 0
    for c in range(O3.num_candidates(g, spec)):
        V, d = O3.candidate(g, spec, state, c)
        if V.size == 0:
            continue
        A = np.eye(len(V)) - Gs[np.ix_(V, V)] * d[None, :]     # FP64 from the stored entries
        b = E[V]
        x64, ok = O.gauss_pp(A, b)
        assert ok
        LU, piv = _lu32(A)
        y0 = _solve32(LU, piv, b).astype(np.complex128)
        r = b - A @ y0                                          # FP64 residual
        dy = _solve32(LU, piv, r).astype(np.complex128)
        y1 = y0 + dy
        scale = np.max(np.abs(x64))
        worst_plain = max(worst_plain, np.max(np.abs(y0 - x64)) / scale)
        worst_ir = max(worst_ir, np.max(np.abs(y1 - x64)) / scale)
        worst_corr = max(worst_corr, np.max(np.abs(np.concatenate([dy.real, dy.imag]))) /
                         np.max(np.abs(np.concatenate([y1.real, y1.imag]))))
        count += 1
    assert count > 10
    print(f"max rel error: FP32 factors {worst_plain:.2e}, + one FP64 refinement {worst_ir:.2e}; "
          f"largest correction {worst_corr:.2e}")
    assert worst_ir <= 1e-12
    assert worst_plain >= 1e-9              # the refinement is what reaches FP64
    assert worst_corr <= 2.0 ** -10 / 100   # far from the singularity flag
