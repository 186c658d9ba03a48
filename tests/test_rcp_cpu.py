"""The pivot reciprocals of the capacitance factorisations (`rcp_nr` and `rcp_nr_i` in
csrc/gf_internal.cuh): Newton's iteration for 1/m on the mantissa m in [1, 2), seeded with the
correctly rounded FP32 reciprocal of m (rcp_nr) or of m truncated to 24 bits (rcp_nr_i, whose
seed is built from bit patterns by integer operations), two steps y <- y + y (1 - m y) with fused
multiply-adds, then an exact power-of-two scaling.  Restated here operation by operation in exact rational arithmetic (each fused
multiply-add rounded once, as the hardware does) and checked against the error bound of the
method: within 1 ulp of 1/v everywhere, correctly rounded for random mantissas (not always: just
above a power of two the result may round to that power)."""
import random
import struct
from fractions import Fraction

import numpy as np
import pytest


def _bits(x: float) -> int:
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _double(b: int) -> float:
    return struct.unpack("<d", struct.pack("<q", b))[0]


def _fma(a: float, b: float, c: float) -> float:
    return float(Fraction(a) * Fraction(b) + Fraction(c))      # exact, then one rounding


def _float(b: int) -> float:
    return float(struct.unpack("<f", struct.pack("<i", b))[0])


def _float_bits(x) -> int:
    return struct.unpack("<i", struct.pack("<f", float(x)))[0]


def rcp_nr(v: float, seed_truncated: bool = False) -> float:
    b = _bits(v)
    e = ((b >> 52) & 0x7FF) - 1023
    m = _double((b & 0x000FFFFFFFFFFFFF) | 0x3FF0000000000000)
    if seed_truncated:
        # rcp_nr_i: FP32 reciprocal of the 24 leading bits of m, its pattern moved into an FP64 one
        yf = np.float32(1.0) / np.float32(_float(0x3F800000 | ((b >> 29) & 0x7FFFFF)))
        fb = _float_bits(yf)
        y = _double(((((fb >> 23) & 0xFF) + (1023 - 127)) << 52) | ((fb & 0x7FFFFF) << 29))
        assert y == float(yf)                                  # the pattern move is exact
    else:
        y = float(np.float32(1.0) / np.float32(m))             # correctly rounded FP32 reciprocal
    r = _fma(-m, y, 1.0)
    y = _fma(y, r, y)
    r = _fma(-m, y, 1.0)
    y = _fma(y, r, y)
    return y * _double((1023 - e) << 52)


@pytest.mark.parametrize("seed_truncated", [False, True])
def test_newton_reciprocal_within_one_ulp_and_correctly_rounded(seed_truncated):
    rng = random.Random(7)
    samples = [rng.uniform(1.0, 2.0) * 2.0 ** rng.randint(-90, 90) for _ in range(4000)]
    # mantissas next to 1 and 2 and exact powers of two
    samples += [2.0 ** k for k in range(-60, 61, 7)]
    samples += [np.nextafter(1.0, 2.0) * 2.0 ** k for k in (-30, 0, 30)]
    samples += [np.nextafter(2.0, 1.0) * 2.0 ** k for k in (-30, 0, 30)]
    rounded = 0
    for i, v in enumerate(samples):
        y = rcp_nr(v, seed_truncated)
        exact = Fraction(1) / Fraction(v)
        ulp = Fraction(float(np.spacing(abs(float(exact)))))
        assert abs(Fraction(y) - exact) <= ulp, (v, y)
        rounded += y == 1.0 / v                               # Python's division rounds correctly
        if i < 4000:
            assert y == 1.0 / v, (v, y)                       # random mantissas: correctly rounded
    assert rounded >= len(samples) - 8
