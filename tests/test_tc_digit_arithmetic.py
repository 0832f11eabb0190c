"""The arithmetic behind the tensor-core contractions, checked against exact
rationals on the CPU.  A float-float value x = hi + lo of a row whose largest
|hi| is below 2^e is split into five signed 9-bit digits,
    x = 2^(e - 8) sum_i d_i 512^(1 - i) + r,   |d_i| <= 256,   |r| <= 2^(e - 45),
each digit the nearest integer to the remainder left by the ones before (its
binary32 low part never rounded); digit products are integers below 2^16, so
the level sums of at most 48 points and 5 plane pairs stay below 2^24 (exact in
binary32); the five level sums of an output are recombined in float-float
(TwoSum of the two leading, the rest into the low part) to better than 2^-42 of
the leading level's scale.  The restatement here follows those rules in
IEEE binary32 (numpy float32, round to nearest per operation; a fused
multiply-add is an exact product and sum rounded once) and imports nothing
from the package or the oracle."""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32
S = 5


def _rne(x):
    M = f32(12582912.0)   # 1.5 * 2^23: (x + M) - M rounds |x| <= 2^22 to an integer
    return f32(f32(x + M) - M)


def _digits(hi, lo, e):
    k = 8 - e
    s1, s2 = f32(2.0 ** min(k, 126)), f32(2.0 ** max(k - 126, 0))
    u, ul = f32(f32(hi * s1) * s2), f32(f32(lo * s1) * s2)
    d = [_rne(u)]
    for _ in range(1, S):
        u = f32(f32(u - d[-1]) * f32(512.0))
        ul = f32(ul * f32(512.0))
        d.append(_rne(f32(u + ul)))
    return d


def _scale_exp(mx):
    if mx == 0:
        return 0
    m, ex = np.frexp(np.float64(mx))   # mx = m 2^ex, 0.5 <= m < 1: mx < 2^ex
    return int(ex)


def _fma32(a, b, c):
    # exact a b + c rounded once to binary32 (the binary64 step between is exact:
    # a b + c here has at most 53 significant bits)
    x = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    assert Fraction(float(x)) == x
    return f32(float(x))


def _combine(acc):
    a, b = f32(acc[0]), f32(f32(acc[1]) * f32(1.0 / 512.0))
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    w = f32(1.0 / 262144.0)
    for l in range(2, S):
        e = _fma32(f32(acc[l]), w, e)
        w = f32(w * f32(1.0 / 512.0))
    t = f32(s + e)
    e = f32(e - f32(t - s))
    return t, e


def _ff(rng, scale):
    hi = f32(rng.uniform(-1, 1) * scale)
    ulp = np.spacing(np.abs(hi)) if hi != 0 else f32(0)
    lo = f32(rng.uniform(-0.5, 0.5) * ulp)
    return hi, lo


@pytest.mark.parametrize("row_exp", [0, 7, -30, -90, -118, 60])
def test_digit_split_bounds_and_remainder(row_exp):
    rng = np.random.default_rng(1000 + row_exp)
    for _ in range(2000):
        # entries of one row: the largest near 2^row_exp, others down to 2^-40 of it
        mag = 2.0 ** (row_exp - rng.integers(0, 40)) * rng.uniform(0.5, 1.0)
        hi, lo = _ff(rng, mag)
        e = _scale_exp(2.0 ** row_exp * 0.99)        # the row's maximum lies below 2^e
        if abs(float(hi)) >= 2.0 ** e:
            continue
        d = _digits(hi, lo, e)
        assert all(abs(float(x)) <= 256 and float(x) == int(x) for x in d)
        val = sum(Fraction(int(x)) * Fraction(512) ** (1 - i) for i, x in enumerate(d, start=1))
        val *= Fraction(2) ** (e - 8)
        exact = Fraction(float(hi)) + Fraction(float(lo))
        assert abs(val - exact) <= Fraction(2) ** (e - 45)


def test_digits_of_a_subnormal_row_and_of_zero():
    hi, lo = f32(3e-39), f32(0.0)                    # binary32 subnormal maximum
    e = -125
    d = _digits(hi, lo, e)
    val = sum(Fraction(int(x)) * Fraction(512) ** (1 - i) for i, x in enumerate(d, start=1)) * Fraction(2) ** (e - 8)
    assert abs(val - Fraction(float(hi))) <= Fraction(2) ** (e - 45)
    assert _digits(f32(0), f32(0), 0) == [0.0] * S


def test_level_sums_stay_exact_in_binary32():
    # level L = i + j sums at most 5 plane pairs over at most 48 points of
    # digit products |d_i d_j| <= 2^16
    bound = 48 * 5 * 256 * 256
    assert bound < 2 ** 24
    rng = np.random.default_rng(7)
    for _ in range(200):
        A = rng.integers(-256, 257, size=(5, 48))
        B = rng.integers(-256, 257, size=(5, 48))
        for L in range(2, S + 2):
            pairs = [(i, L - i) for i in range(1, S + 1) if 1 <= L - i <= S]
            exact = sum(int(np.dot(A[i - 1], B[j - 1])) for i, j in pairs)
            acc = f32(0)
            for i, j in pairs:                       # any order of binary32 additions of integers < 2^24
                for q in range(48):
                    acc = f32(acc + f32(int(A[i - 1, q]) * int(B[j - 1, q])))
            assert int(acc) == exact


def test_level_combination_error():
    rng = np.random.default_rng(11)
    worst = Fraction(0)
    for _ in range(3000):
        acc = [f32(int(rng.integers(-(2 ** 23), 2 ** 23))) for _ in range(S)]
        s, e = _combine(acc)
        exact = sum(Fraction(int(a)) * Fraction(512) ** (-l) for l, a in enumerate(acc))
        err = abs(Fraction(float(s)) + Fraction(float(e)) - exact)
        assert abs(float(e)) <= float(np.spacing(abs(s))) / 2 + 1e-300
        worst = max(worst, err / Fraction(2 ** 24))   # relative to the leading level's scale
    assert worst <= Fraction(2) ** -42


def test_products_of_split_operands():
    """A product of two split values, with the plane pairs i + j > 6 left out,
    is within ~2^-42 of the product of the two scales."""
    rng = np.random.default_rng(3)
    for _ in range(2000):
        (ha, la), (hb, lb) = _ff(rng, 0.9), _ff(rng, 0.9)
        da, db = _digits(ha, la, 0), _digits(hb, lb, 0)
        kept = Fraction(0)
        for i in range(1, S + 1):
            for j in range(1, S + 1):
                if i + j <= S + 1:
                    kept += Fraction(int(da[i - 1]) * int(db[j - 1])) * Fraction(512) ** (2 - i - j)
        kept *= Fraction(2) ** -16
        exact = (Fraction(float(ha)) + Fraction(float(la))) * (Fraction(float(hb)) + Fraction(float(lb)))
        assert abs(kept - exact) <= Fraction(2) ** -42
