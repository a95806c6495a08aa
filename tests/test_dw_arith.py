"""Host-side check of the double-word arithmetic recipe the double-word steps
use (fp64 values carried as hi + lo float pairs): the conversion from fp64,
the row sum of products collected as (s, e) with TwoSum and exact product
errors, and the renormalised x + g v update, written out here with numpy
float32 operations (each rounds to nearest, as the device's __fadd_rn,
__fmul_rn, __fmaf_rn do) and compared with exact rational arithmetic.

These fix the accuracy the kernels' documentation states: a few units of
2^-48 relative to the magnitudes of the terms (2^-53 for native fp64)."""
from fractions import Fraction

import numpy as np

f32 = np.float32
U48 = 2.0 ** -48


def fl(x):
    return f32(x)


def fma32(a, b, c):
    # a b is exact in float64 (two 24-bit significands); the sum rounds once
    # in float64 and once to float32 (the second rounding is exact whenever
    # the result is an error term that fits in 24 bits)
    return fl(np.float64(a) * np.float64(b) + np.float64(c))


def two_sum(a, b):
    s = fl(a + b)
    bv = fl(s - a)
    return s, fl(fl(a - fl(s - bv)) + fl(b - bv))


def dw_mac(s, e, ah, al, bh, bl):
    p = fl(ah * bh)
    pe = fma32(ah, bh, -p)
    pe = fma32(ah, bl, pe)
    pe = fma32(al, bh, pe)
    t, err = two_sum(s, p)
    return t, fl(e + fl(err + pe))


def dw_axpy(xh, xl, gh, gl, vh, vl):
    p = fl(gh * vh)
    pe = fma32(gh, vh, -p)
    pe = fma32(gh, vl, pe)
    pe = fma32(gl, vh, pe)
    t, err = two_sum(xh, p)
    lo = fl(xl + fl(pe + err))
    h = fl(t + lo)
    return h, fl(lo - fl(h - t))


def split(x):
    h = fl(x)
    return h, fl(np.float64(x) - np.float64(h))


def exact(h, l):
    return Fraction(float(h)) + Fraction(float(l))


def test_two_sum_is_exact():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        a, b = fl(rng.standard_normal() * 10.0 ** rng.integers(-8, 8)), fl(rng.standard_normal())
        s, e = two_sum(a, b)
        assert Fraction(float(s)) + Fraction(float(e)) == Fraction(float(a)) + Fraction(float(b))


def test_conversion_keeps_48_bits():
    rng = np.random.default_rng(2)
    for x in rng.standard_normal(2000) * 10.0 ** rng.integers(-6, 6, 2000):
        h, l = split(x)
        assert abs(exact(h, l) - Fraction(float(x))) <= Fraction(U48) * abs(Fraction(float(x)))


def test_row_sum_within_a_few_units_of_2_48():
    """13 products (a Topi row) added to a start value, with cancellation:
    the error stays below 8 units of 2^-48 of the sum of the magnitudes."""
    rng = np.random.default_rng(3)
    worst = 0.0
    for _ in range(3000):
        a = [split(x) for x in rng.standard_normal(13)]
        v = [split(x) for x in rng.standard_normal(13)]
        w = split(rng.standard_normal())
        s, e = fl(-w[0]), fl(-w[1])
        for (ah, al), (vh, vl) in zip(a, v):
            s, e = dw_mac(s, e, ah, al, vh, vl)
        h, l = two_sum(s, e)
        ref = -exact(*w) + sum(exact(*x) * exact(*y) for x, y in zip(a, v))
        mag = abs(exact(*w)) + sum(abs(exact(*x) * exact(*y)) for x, y in zip(a, v))
        rel = float(abs(exact(h, l) - ref) / mag)
        worst = max(worst, rel)
    assert worst < 8 * U48, worst / U48


def test_axpy_within_a_few_units_of_2_48():
    rng = np.random.default_rng(4)
    worst = 0.0
    for _ in range(3000):
        x, g, v = split(rng.standard_normal()), split(rng.standard_normal() * 0.1), split(rng.standard_normal())
        h, l = dw_axpy(*x, *g, *v)
        ref = exact(*x) + exact(*g) * exact(*v)
        mag = abs(exact(*x)) + abs(exact(*g) * exact(*v))
        worst = max(worst, float(abs(exact(h, l) - ref) / mag))
    assert worst < 8 * U48, worst / U48


def test_planted_mistake_loses_accuracy():
    """Without the product's rounding error (a plain float product) the same
    row sum is only accurate to about 2^-24: the check above can fail."""
    rng = np.random.default_rng(5)
    a = [split(x) for x in rng.standard_normal(13)]
    v = [split(x) for x in rng.standard_normal(13)]
    s, e = f32(0), f32(0)
    for (ah, al), (vh, vl) in zip(a, v):
        t, err = two_sum(s, fl(ah * vh))
        s, e = t, fl(e + err)
    ref = sum(exact(*x) * exact(*y) for x, y in zip(a, v))
    mag = sum(abs(exact(*x) * exact(*y)) for x, y in zip(a, v))
    assert float(abs(exact(*two_sum(s, e)) - ref) / mag) > 8 * U48
