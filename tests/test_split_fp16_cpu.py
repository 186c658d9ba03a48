"""The split-FP16 arithmetic of the complex64 rank-k p update (`f16_split`, `scale_exp` and the
three products per K chunk in csrc/gf_update_c64.cu), restated in numpy.

A row of A' (a column of B') is scaled by 2^(14 - E), with E the smallest exponent such that
every |x| of the row lies below 2^E, so that every scaled x' lies in (-2^14, 2^14).  Then
x' = hi + lo + r with hi = fp16(x') and lo = fp16(x' - hi), where x' - hi is exact in FP32.  The
update accumulates hi_a hi_b + hi_a lo_b + lo_a hi_b over K in FP32; those products are exact
(11 x 11 bits).  The error of one product against a' b' is lo_a lo_b + r_a b' + r_b a'.  With
|lo| <= 2^-11 |x'| and |r| <= 2^-11 |lo| while lo is a normal FP16 (else |r| <= 2^-25, half the
FP16 subnormal step), that error is at most 3 2^-22 |a'||b'| + 2^-25 (|a'| + |b'|) + 2^-50 (the
last term is r_a r_b when both operands lie below the FP16 normal range).  The
accumulation is modelled as 3K FP32 additions, each with a relative error of at most 2^-23 of
the running sum of magnitudes, which covers rounding to nearest and toward zero alike."""
import numpy as np

F32 = np.float32


def scale_exp(m: float) -> int:
    return int(np.frexp(np.float32(m))[1]) if m > 0 else 0         # smallest E with m < 2^E


def split(xs: np.ndarray):
    hi = xs.astype(np.float16)
    diff = xs - hi.astype(F32)
    assert np.array_equal(diff.astype(np.float64), xs.astype(np.float64) - hi.astype(np.float64))
    return hi, diff.astype(np.float16)


def scaled(v: np.ndarray) -> np.ndarray:
    E = scale_exp(float(np.max(np.abs(v))))
    xs = (v * F32(2.0 ** (14 - E))).astype(F32)
    assert np.all(np.abs(xs) < 2.0 ** 14)
    return xs


def dot_split(a: np.ndarray, b: np.ndarray):
    ap, bp = scaled(a), scaled(b)
    ha, la = split(ap)
    hb, lb = split(bp)
    h = lambda v: v.astype(F32)
    acc = F32(0.0)
    for k in range(a.size):
        for t in (h(ha[k]) * h(hb[k]), h(ha[k]) * h(lb[k]), h(la[k]) * h(hb[k])):
            acc = F32(acc + F32(t))
    a64, b64 = ap.astype(np.float64), bp.astype(np.float64)
    prod = (h(ha).astype(np.float64) * h(hb) + h(ha).astype(np.float64) * h(lb)
            + h(la).astype(np.float64) * h(hb))
    return a64, b64, prod, float(acc)


def _cases(rng, n, wide):
    for _ in range(n):
        K = int(rng.choice([8, 32, 96, 256]))
        if wide:                                    # magnitudes spread over 2^40
            ma, mb = 2.0 ** rng.uniform(-30, 10, K), 2.0 ** rng.uniform(-30, 10, K)
        else:                                       # every entry within 2^-17 of its row's largest
            ma, mb = 2.0 ** rng.uniform(-6, 0, K), 2.0 ** rng.uniform(-6, 0, K)
        yield (rng.uniform(-1, 1, K) * ma).astype(F32), (rng.uniform(-1, 1, K) * mb).astype(F32)


def test_per_product_and_accumulated_bounds():
    rng = np.random.default_rng(5)
    worst = 0.0
    for wide in (False, True):
        for a, b in _cases(rng, 600, wide):
            a64, b64, prod, acc = dot_split(a, b)
            per = (3 * 2.0 ** -22 * np.abs(a64) * np.abs(b64) + 2.0 ** -25 * (np.abs(a64) + np.abs(b64))
                   + 2.0 ** -50)
            assert np.all(np.abs(a64 * b64 - prod) <= per)
            S = float(np.sum(np.abs(a64) * np.abs(b64)))
            bound = float(np.sum(per)) + 3 * a.size * 2.0 ** -23 * S
            err = abs(acc - float(np.dot(a64, b64)))
            assert err <= bound
            worst = max(worst, err / bound)
    assert worst > 0.05                             # the bound is not vacuous


def test_error_relative_to_the_sum_of_magnitudes_when_entries_are_comparable():
    """Entries within 2^-17 of their row's (column's) largest keep lo normal: the error is then
    relative to sum |a'||b'|, at most 3 2^-22 + 3K 2^-23 of it (K <= 256), and far smaller in
    practice (median below 2^-22)."""
    rng = np.random.default_rng(7)
    rel = []
    for a, b in _cases(rng, 800, wide=False):
        a64, b64, _, acc = dot_split(a, b)
        S = float(np.sum(np.abs(a64) * np.abs(b64)))
        r = abs(acc - float(np.dot(a64, b64))) / S
        assert r <= 3 * 2.0 ** -22 + 3 * a.size * 2.0 ** -23
        rel.append(r)
    assert np.median(rel) < 2.0 ** -22


def test_absolute_term_dominates_only_for_entries_far_below_their_rows_largest():
    """A row whose large entries meet the column's small ones: relative to sum |a'||b'| the error
    can be large, but it stays within the absolute 2^-25 (|a'| + |b'|) terms, i.e. about 2^-39 of
    the product of the two largest magnitudes per product."""
    K = 8
    a = np.array([1.0] + [2.0 ** -30] * (K - 1), dtype=F32)
    b = np.array([2.0 ** -30] + [1.0 / 3.0] * (K - 1), dtype=F32)
    a64, b64, prod, acc = dot_split(a, b)
    err = abs(acc - float(np.dot(a64, b64)))
    assert err <= float(np.sum(2.0 ** -25 * (np.abs(a64) + np.abs(b64)) + 3 * 2.0 ** -22 * np.abs(a64 * b64)
                               + 2.0 ** -50)) \
        + 3 * K * 2.0 ** -23 * float(np.sum(np.abs(a64 * b64)))
    assert err <= K * 2.0 ** -39 * float(np.max(np.abs(a64)) * np.max(np.abs(b64))) * 2
