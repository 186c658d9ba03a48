"""The digit decomposition of the FP64-accurate tensor-core update (`oz_digits_i` and
`oz_exponent_bits` in csrc/gf_stage_bodies.cuh), restated operation by operation in Python
integers, against the FP64 sequence it stands for (d_a = rint(r_a 2^(9(a+1))), r_(a+1) = r_a -
d_a 2^(-9(a+1)), every step exact, so exact rationals model it) and against what the update
needs: six digits, the first within +-512 and the others within +-256 (exact in TF32), summing to
x = v 2^-E rounded to a multiple of 2^-54 (ties to even), with E the smallest exponent such that
every |v| of the row lies below 2^E."""
import math
import random
import struct
from fractions import Fraction

import numpy as np

W, S = 9, 6                      # bits per digit, digits per value


def _bits(x: float) -> int:
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _rne_shift(x: int, s: int) -> int:
    """x / 2^s rounded to the nearest integer, ties to even, as the kernel forms it with an
    arithmetic shift: (x + 2^(s-1) - 1 + ((x >> s) & 1)) >> s."""
    return (x + (1 << (s - 1)) - 1 + ((x >> s) & 1)) >> s


def digits_int(v: float, E: int, trace=None):
    b = _bits(v)
    ef = (b >> 52) & 0x7FF
    M = (b & 0x000FFFFFFFFFFFFF) | (0x0010000000000000 if ef else 0)
    sh = (ef if ef else 1) - 1075 + 54 - E
    if sh >= 0:
        X = M << min(sh, 63)
    elif sh > -54:
        s = -sh
        q, rem, half = M >> s, M & ((1 << s) - 1), 1 << (s - 1)
        X = q + (1 if (rem > half or (rem == half and (q & 1))) else 0)
    else:
        X = 0
    if b < 0:
        X = -X
    d = []
    for a in range(S - 1):
        sft = 45 - W * a
        if trace is not None:
            trace.append(X % (1 << sft) == 1 << (sft - 1))      # the remainder is an exact tie
        da = _rne_shift(X, sft)
        d.append(da)
        X -= da << sft
    d.append(X)
    return d


def _rint(q: Fraction) -> int:
    f = math.floor(q)
    r = q - f
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and f % 2 == 1):
        return f + 1
    return f


def digits_fp64(v: float, E: int):
    r = Fraction(v) / Fraction(2) ** E
    d = []
    for a in range(S):
        t = _rint(r * 2 ** (W * (a + 1)))
        d.append(t)
        r -= Fraction(t, 2 ** (W * (a + 1)))
    return d


def exponent_bits(mb: int) -> int:
    if mb <= 0:
        return 0
    ef = mb >> 52
    return (ef - 1023 if ef else (mb.bit_length() - 1) - 1074) + 1


def _exponent_ref(m: float) -> int:
    """Smallest E with m < 2^E (m > 0): frexp gives m = f 2^e with f in [0.5, 1)."""
    return math.frexp(m)[1] if m > 0 else 0


def _row(rng, n):
    scale = 2.0 ** rng.randint(-60, 60)
    return [rng.uniform(-1.0, 1.0) * scale * (2.0 ** -rng.randint(0, 40) if rng.random() < 0.3 else 1.0)
            for _ in range(n)]


def test_exponent_of_the_row_maximum():
    rng = random.Random(3)
    vals = [0.0, 5e-324, 2.2250738585072014e-308, 1.0, 0.5, np.nextafter(1.0, 0.0), 1e300]
    vals += [rng.uniform(0, 1) * 2.0 ** rng.randint(-1070, 1000) for _ in range(2000)]
    for m in vals:
        E = exponent_bits(_bits(m) & 0x7FFFFFFFFFFFFFFF)
        assert E == _exponent_ref(m), m
        if m > 0:
            assert m < 2.0 ** E and m >= 2.0 ** (E - 1)


def test_integer_digits_sum_ranges_and_agreement_with_the_fp64_sequence():
    rng = random.Random(11)
    differ = values = 0
    for _ in range(1500):
        row = _row(rng, 8)
        E = exponent_bits(max(_bits(v) & 0x7FFFFFFFFFFFFFFF for v in row))
        for v in row:
            di = digits_int(v, E)
            df = digits_fp64(v, E)
            x = Fraction(v) / Fraction(2) ** E
            assert abs(x) < 1
            assert abs(di[0]) <= 512 and all(abs(t) <= 256 for t in di[1:]), di
            total = sum(Fraction(t, 2 ** (W * (a + 1))) for a, t in enumerate(di))
            assert total == Fraction(_rint(x * 2 ** 54), 2 ** 54)          # x rounded at 2^-54
            assert total == sum(Fraction(t, 2 ** (W * (a + 1))) for a, t in enumerate(df))
            if di != df:
                # the sequences part where the rounded value meets an exact tie of a digit that
                # the exact value does not (the FP64 sequence sees the bits below 2^-54)
                tr = []
                digits_int(v, E, tr)
                first = next(a for a in range(S) if di[a] != df[a])
                assert first < S - 1 and tr[first], (v, E, di, df)
                assert _rint(x * 2 ** 54) != x * 2 ** 54
                differ += 1
            values += 1
    assert differ < values // 200


def test_ties_and_edges():
    # exact ties at a digit boundary round to even in both forms; zero and tiny values
    for k in range(-6, 7):
        v = (k + 0.5) * 2.0 ** -9
        assert digits_int(v, 0) == digits_fp64(v, 0)
        assert digits_int(v, 0)[0] % 2 == 0
    assert digits_int(0.0, 0) == [0] * S and digits_int(-0.0, 5) == [0] * S
    assert digits_int(2.0 ** -60, 0) == [0] * S                           # below half a unit
    assert digits_int(3 * 2.0 ** -56, 0)[-1] == 1                          # 0.75 unit rounds up
    v = math.ldexp(1.0, -1070)                                             # subnormal row maximum
    E = exponent_bits(_bits(v))
    assert digits_int(v, E) == digits_fp64(v, E)
    # a value within 2^-54 of an earlier digit's tie: the sums agree, the digits may not
    v = (3 + 0.5) * 2.0 ** -9 + 2.0 ** -70
    di, df = digits_int(v, 0), digits_fp64(v, 0)
    assert sum(Fraction(t, 2 ** (W * (a + 1))) for a, t in enumerate(di)) == \
        sum(Fraction(t, 2 ** (W * (a + 1))) for a, t in enumerate(df))
