"""The integer widening of FP32 to FP64 in the complex64 row gather (`f2d_bits` in
csrc/gf_update_c64.cu), restated in Python: the result must be the exact FP64 value of the
float (IEEE conversion is exact for every finite float), bit for bit, for normals, subnormals,
signed zeros and infinities; a NaN stays a NaN of the same sign."""
import math
import random
import struct

import numpy as np


def f2d_bits(b: int) -> int:
    """b: the float's 32 bits; returns the double's 64 bits."""
    e, m = (b >> 23) & 0xFF, b & 0x7FFFFF
    s = (b >> 31) << 63
    if e == 0xFF:
        return s | 0x7FF0000000000000 | (m << 29)
    if e != 0:
        return s | ((e + (1023 - 127)) << 52) | (m << 29)
    if m == 0:
        return s
    t = m.bit_length() - 1                                  # 31 - clz(m)
    return s | ((t - 149 + 1023) << 52) | ((m << (52 - t)) & 0x000FFFFFFFFFFFFF)


def _ref_bits(b: int) -> int:
    f = np.array([b], dtype=np.uint32).view(np.float32)[0]
    return int(np.array([np.float64(f)]).view(np.uint64)[0])


def test_finite_and_infinite_floats_widen_exactly():
    rng = random.Random(29)
    cases = [0, 1, 2, 0x3FFFFF, 0x400000, 0x7FFFFF, 0x800000, 0x3F800000, 0x7F7FFFFF, 0x7F800000]
    cases += [rng.getrandbits(23) for _ in range(20000)]                              # subnormals
    cases += [(rng.randint(1, 254) << 23) | rng.getrandbits(23) for _ in range(20000)]  # normals
    for b in cases:
        for sign in (0, 1 << 31):
            bb = b | sign
            assert f2d_bits(bb) == _ref_bits(bb), hex(bb)
    # every subnormal's value is m 2^-149 exactly
    for m in (1, 3, 0x12345, 0x7FFFFF):
        d = struct.unpack("<d", struct.pack("<Q", f2d_bits(m)))[0]
        assert d == math.ldexp(m, -149)


def test_nan_stays_nan_with_its_sign():
    for b in (0x7FC00000, 0x7F800001, 0x7FFFFFFF, 0xFFC00000, 0xFF800001):
        d = struct.unpack("<d", struct.pack("<Q", f2d_bits(b)))[0]
        assert math.isnan(d)
        assert (f2d_bits(b) >> 63) == (b >> 31)
