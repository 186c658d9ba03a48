"""The integer keys of the selection kernels (`ord_key`, `key_value` in
csrc/gf_stage_bodies.cuh), restated in Python.  A dFOM value's key is its IEEE-754 bit pattern
as a signed 64-bit integer, with the magnitude bits of negative values inverted, -0 mapped to +0
and every NaN to the smallest integer.  Comparing keys must order values exactly as comparing
the doubles does, equal values must share a key, and key_value must give the value back."""
import math
import random
import struct

LLONG_MIN = -(1 << 63)
MAG = 0x7FFFFFFFFFFFFFFF


def _bits(v: float) -> int:
    return struct.unpack("<q", struct.pack("<d", v))[0]


def _double(b: int) -> float:
    return struct.unpack("<d", struct.pack("<q", b))[0]


def ord_key(v: float) -> int:
    b = _bits(v)
    if (b & MAG) > 0x7FF0000000000000:
        return LLONG_MIN
    if b == LLONG_MIN:                       # -0
        b = 0
    return b if b >= 0 else b ^ MAG


def key_value(k: int) -> float:
    return _double(k if k >= 0 else k ^ MAG)


def _values(rng, n):
    vals = [0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, -2.2250738585072014e-308,
            1.0, -1.0, math.inf, -math.inf, 1.7976931348623157e308, -1.7976931348623157e308]
    for _ in range(n):
        m = rng.random()
        v = m * 2.0 ** rng.randint(-1074, 1023)
        vals.append(v if rng.random() < 0.5 else -v)
    vals += [vals[i] for i in range(0, len(vals), 7)]          # repeats: equal values
    return vals


def test_keys_order_like_the_doubles():
    rng = random.Random(17)
    vals = _values(rng, 4000)
    for _ in range(20000):
        a, b = rng.choice(vals), rng.choice(vals)
        ka, kb = ord_key(a), ord_key(b)
        assert (ka < kb) == (a < b), (a, b)
        assert (ka == kb) == (a == b), (a, b)
    assert ord_key(-0.0) == ord_key(0.0) == 0
    assert ord_key(-math.inf) > LLONG_MIN


def test_nan_is_below_everything_and_values_round_trip():
    rng = random.Random(19)
    for nan_bits in (0x7FF8000000000000, 0x7FF0000000000001, -0x0008000000000000, -1):
        v = _double(nan_bits)
        assert math.isnan(v)
        assert ord_key(v) == LLONG_MIN
        assert ord_key(v) < ord_key(-math.inf)
    for v in _values(rng, 3000):
        r = key_value(ord_key(v))
        assert r == v
        if v != 0.0:
            assert _bits(r) == _bits(v)
        else:
            assert _bits(r) == 0                                  # -0 comes back as +0


def test_the_greedy_choice_on_keys_equals_the_double_scan():
    """max by (key, lowest id) over an array equals the scan on doubles that keeps the first
    largest value, NaN never chosen while a number is present."""
    rng = random.Random(23)
    for _ in range(300):
        n = rng.randint(1, 60)
        d = [rng.choice([rng.uniform(-1, 1), 0.0, -0.0, -math.inf, float("nan"), 0.5]) for _ in range(n)]
        bk, bid = ord_key(-math.inf), 1 << 62
        for i, v in enumerate(d):
            k = ord_key(v)
            if k > bk or (k == bk and i < bid):
                bk, bid = k, i
        finite = [(v, i) for i, v in enumerate(d) if not math.isnan(v)]
        if finite:
            best = max(v for v, _ in finite)
            want = min(i for v, i in finite if v == best)
            assert bid == want and key_value(bk) == best
