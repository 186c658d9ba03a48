"""The pivot reciprocal of the capacitance factorisations (`rcp_nr` in csrc/gf_internal.cuh):
Newton's iteration for 1/m on the mantissa m in [1, 2), seeded with the correctly rounded FP32
reciprocal, two steps y <- y + y (1 - m y) with fused multiply-adds, then an exact power-of-two
scaling.  Restated here operation by operation in exact rational arithmetic (each fused
multiply-add rounded once, as the hardware does) and checked against the error bound of the
method: within 1 ulp of 1/v everywhere, correctly rounded for random mantissas (not always: just
above a power of two the result may round to that power)."""
import random
import struct
from fractions import Fraction

import numpy as np


def _bits(x: float) -> int:
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _double(b: int) -> float:
    return struct.unpack("<d", struct.pack("<q", b))[0]


def _fma(a: float, b: float, c: float) -> float:
    return float(Fraction(a) * Fraction(b) + Fraction(c))      # exact, then one rounding


def rcp_nr(v: float) -> float:
    b = _bits(v)
    e = ((b >> 52) & 0x7FF) - 1023
    m = _double((b & 0x000FFFFFFFFFFFFF) | 0x3FF0000000000000)
    y = float(np.float32(1.0) / np.float32(m))                 # correctly rounded FP32 reciprocal
    r = _fma(-m, y, 1.0)
    y = _fma(y, r, y)
    r = _fma(-m, y, 1.0)
    y = _fma(y, r, y)
    return y * _double((1023 - e) << 52)


def test_newton_reciprocal_within_one_ulp_and_correctly_rounded():
    rng = random.Random(7)
    samples = [rng.uniform(1.0, 2.0) * 2.0 ** rng.randint(-90, 90) for _ in range(4000)]
    # mantissas next to 1 and 2 and exact powers of two
    samples += [2.0 ** k for k in range(-60, 61, 7)]
    samples += [np.nextafter(1.0, 2.0) * 2.0 ** k for k in (-30, 0, 30)]
    samples += [np.nextafter(2.0, 1.0) * 2.0 ** k for k in (-30, 0, 30)]
    rounded = 0
    for i, v in enumerate(samples):
        y = rcp_nr(v)
        exact = Fraction(1) / Fraction(v)
        ulp = Fraction(float(np.spacing(abs(float(exact)))))
        assert abs(Fraction(y) - exact) <= ulp, (v, y)
        rounded += y == 1.0 / v                               # Python's division rounds correctly
        if i < 4000:
            assert y == 1.0 / v, (v, y)                       # random mantissas: correctly rounded
    assert rounded >= len(samples) - 8
