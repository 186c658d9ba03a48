"""The epilogue arithmetic of the FP64-accurate tensor-core update (`oz_combine` and
`oz_to_double` in csrc/gf_update_tc.cu), restated operation by operation in Python integers.

Each level's FP32 accumulator receives the integer digit products of its level (digits within
+-512 for the first, +-256 for the others; K = 8).  What the update needs from that arithmetic:
  * every partial sum, in any order of the products, is an integer of magnitude at most 2^22,
    exact in FP32 whatever the order or rounding of the additions; adding 1.5 * 2^23 gives an
    integer in [2^23, 2^24], also exact, whose bit pattern minus that of 1.5 * 2^23 is the sum;
  * the three int32 joins of adjacent levels do not overflow, and the int64 recombination is
    sum_L acc_L 2^(9 (5 - L)) in units of 2^-63, rounded (half up) to units of 2^-59;
  * the integer-built double is D 2^u with the 53-bit significand truncated toward zero."""
import random
import struct
from fractions import Fraction

import numpy as np

LV, K = 6, 8
BIAS_BITS = 0x4B400000                       # 1.5 * 2^23
BIAS = np.float32(12582912.0)
MASK64 = (1 << 64) - 1


def _f32_bits(x: np.float32) -> int:
    return int(np.array([x], dtype=np.float32).view(np.int32)[0])


def combine(level_bits):
    """oz_combine on the six accumulator bit patterns; returns D (units 2^-59) and the joins."""
    b = [x - BIAS_BITS for x in level_bits]
    P1 = (b[0] << 9) + b[1]
    P2 = (b[2] << 9) + b[3]
    P3 = (b[4] << 9) + b[5]
    D = (P1 << 32) + (P2 << 14) + ((P3 + 8) >> 4)
    return D, (P1, P2, P3)


def to_double(D: int, u: int) -> float:
    """oz_to_double: two's-complement 64-bit steps of the kernel (its D == 0 test is the case
    lz == 64 here)."""
    sg = -1 if D < 0 else 0
    M = ((D ^ sg) - sg) & MASK64
    lz = 64 - M.bit_length()
    M = (M << (lz & 63)) & MASK64
    mant = M >> 11
    e = 63 - lz + u
    bits = (((e + 1022) << 52) + mant) & MASK64
    if sg:
        bits |= 1 << 63
    return struct.unpack("<d", struct.pack("<Q", bits if lz < 64 else 0))[0]


def _digits(rng, first: bool):
    lim = 512 if first else 256
    return [rng.randint(-lim, lim) for _ in range(K)]


def _levels_fp32(A, B, order):
    """Accumulate each level in FP32 from 0 over its (a, b, k) products in `order`."""
    acc = [np.float32(0.0)] * LV
    for a, b, k in order:
        acc[a + b] = np.float32(acc[a + b] + np.float32(A[a][k] * B[b][k]))
    return acc


def _exact_levels(A, B):
    return [sum(A[a][k] * B[L - a][k] for a in range(L + 1) for k in range(K)) for L in range(LV)]


def test_levels_and_their_biased_bit_patterns_are_exact_in_any_order():
    rng = random.Random(5)
    terms = [(a, b, k) for a in range(LV) for b in range(LV) if a + b < LV for k in range(K)]
    cases = []
    for _ in range(300):
        cases.append(([_digits(rng, a == 0) for a in range(LV)], [_digits(rng, b == 0) for b in range(LV)]))
    # the extreme: every digit at its bound with one sign, so that level 5 reaches 2^22
    ext = [[512] * K] + [[256] * K] * (LV - 1)
    cases += [(ext, ext), (ext, [[-x for x in row] for row in ext])]
    for A, B in cases:
        exact = _exact_levels(A, B)
        assert max(abs(v) for v in exact) <= 1 << 22
        for trial in range(3):
            order = list(terms)
            random.Random(trial).shuffle(order)
            acc = _levels_fp32(A, B, order)
            for L in range(LV):
                assert float(acc[L]) == exact[L]
                biased = np.float32(acc[L] + BIAS)
                assert 2.0 ** 23 <= float(biased) <= 2.0 ** 24
                assert _f32_bits(biased) - BIAS_BITS == exact[L]
        # the same sums accumulated from 1.5 * 2^23 instead (the bias first): still exact
        for L in range(LV):
            part = BIAS
            for a in range(L + 1):
                for k in range(K):
                    part = np.float32(part + np.float32(A[a][k] * B[L - a][k]))
            assert _f32_bits(part) - BIAS_BITS == exact[L]
    # the worst case level 5 lands on 2^24 itself, whose pattern still decodes to +2^22
    assert _f32_bits(np.float32(2.0 ** 24)) - BIAS_BITS == 1 << 22
    assert _f32_bits(np.float32(2.0 ** 23)) - BIAS_BITS == -(1 << 22)


def test_recombination_fits_int32_joins_and_int64():
    rng = random.Random(9)
    ext = [1 << 21, 1 << 21, (1 << 21) + (1 << 19), (1 << 21) + (1 << 20), (1 << 21) + 3 * (1 << 19), 1 << 22]
    cases = [ext, [-v for v in ext], [0] * LV]
    cases += [[rng.randint(-e, e) for e in ext] for _ in range(3000)]
    for lv in cases:
        bits = [BIAS_BITS + v for v in lv]
        D, (P1, P2, P3) = combine(bits)
        for P in (P1, P2, P3):
            assert -(1 << 31) <= P < (1 << 31)
        exact63 = sum(v << (9 * (LV - 1 - L)) for L, v in enumerate(lv))     # units 2^-63
        assert D == (exact63 + 8) >> 4                                          # half up at 2^-59
        # int64 without overflow, and its negation too (the digit bounds alone allow a little
        # over 2^62; values of magnitude below 1 keep |D| below 8 * 2^59 = 2^62)
        assert abs(D) < (1 << 63) - 1


def test_integer_built_double_truncates_toward_zero():
    rng = random.Random(13)
    Ds = [0, 1, -1, 2, -3, (1 << 53) - 1, 1 << 53, (1 << 53) + 1, -(1 << 53) - 1, (1 << 62) - 1, -(1 << 62) + 1]
    Ds += [rng.randint(-(1 << 62) + 1, (1 << 62) - 1) >> rng.randint(0, 61) for _ in range(5000)]
    for D in Ds:
        u = rng.randint(-900, 900)
        r = to_double(D, u)
        m = abs(D)
        s = max(0, m.bit_length() - 53)
        want = Fraction((m >> s) << s) * Fraction(2) ** u
        if D < 0:
            want = -want
        assert Fraction(r) == want, (D, u)
        assert not (D == 0 and struct.pack("<d", r) != struct.pack("<d", 0.0))    # +0, not -0
