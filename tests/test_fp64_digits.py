"""The arithmetic of the FP64 tensor-core products (op_fp64_gemm = OP_GEMM_TC), emulated
on the CPU with exact integers (no GPU).

A value a of a contraction row with exponent e (max |a| < 2^e) becomes the integer
X = round(a 2^(55 - e)) (half away from zero), written in balanced base 256 as seven
digits d_0..d_6 (d_1..d_6 in [-128, 127], d_0 in [-128, 128]).  A product of two rows
keeps the 28 digit pairs with s + t <= 6, summed per level l = s + t over runs of 256
terms in FP32 (levels 0..3 are exact there); the levels are combined in int64 as
hi = L0 2^24 + L1 2^16 + L2 2^8 + L3, lo = L4 2^16 + L5 2^8 + L6 and scaled back by
2^(e_a + e_b - 62).  These tests check each claim against exact rational arithmetic.
"""
import math
from fractions import Fraction

import numpy as np
import pytest


def to_int(a, e, nd=7):
    """round(a 2^(8 nd - 1 - e)), ties away from zero, exactly (a is a float, |a| < 2^e)."""
    num, den = float(a).as_integer_ratio()
    sgn = -1 if num < 0 else 1
    num = abs(num)
    sh = 8 * nd - 1 - e
    if sh >= 0:
        num <<= sh
    else:
        den <<= -sh
    return sgn * ((2 * num + den) // (2 * den))


def digits(X, nd=7):
    d = [0] * nd
    for s in range(nd - 1, 0, -1):
        lo8 = X & 0xFF
        dd = lo8 - 256 if lo8 >= 128 else lo8
        d[s] = dd
        X = (X - dd) >> 8
    d[0] = X
    return d


def exponent(mx):
    return math.frexp(mx)[1] if mx > 0 else 0


def emulate_dot(a, b, run=256, nd=7):
    """The kernel's product of two contraction rows, with FP32 level sums per run."""
    ea, eb = exponent(np.abs(a).max()), exponent(np.abs(b).max())
    da = [digits(to_int(x, ea, nd), nd) for x in a]
    db = [digits(to_int(x, eb, nd), nd) for x in b]
    hi = lo = 0
    for k0 in range(0, len(a), run):
        L = [np.float32(0.0)] * nd
        for k in range(k0, min(k0 + run, len(a))):
            for s in range(nd):
                for t in range(nd - s):
                    L[s + t] = np.float32(L[s + t] + np.float32(da[k][s] * db[k][t]))
        Li = [int(v) for v in L]
        hi += (Li[0] << 24) + (Li[1] << 16) + (Li[2] << 8) + Li[3]
        lo += sum(Li[lv] << (8 * (nd - 1 - lv)) for lv in range(4, nd))
    assert abs(hi) < 2 ** 63 and abs(lo) < 2 ** 63
    B = 8 * nd - 1
    return math.ldexp(float(hi) * 2.0 ** (8 * (nd - 4)) + float(lo),
                      ea + eb - 2 * B + 8 * (nd - 1)), da, db


def test_digits_reconstruct_the_integer_exactly():
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.standard_normal(300), rng.standard_normal(50) * 1e-12,
                           [0.0, -0.0, 5e-324, 1.0 - 2.0 ** -53, -(1.0 - 2.0 ** -53)]])
    e = exponent(np.abs(vals).max())
    for a in vals:
        X = to_int(a, e)
        assert abs(X) <= 2 ** 55
        d = digits(X)
        assert all(-128 <= v <= 127 for v in d[1:]) and -128 <= d[0] <= 128
        assert sum(v << (8 * (6 - s)) for s, v in enumerate(d)) == X
        # every digit is exactly a BF16 value (8 significant bits)
        assert all(abs(v) < 256 for v in d)
        # rounding a to X costs at most half a unit of 2^(e - 55)
        assert abs(Fraction(a) - Fraction(X) * Fraction(2) ** (e - 55)) <= \
            Fraction(1, 2) * Fraction(2) ** (e - 55)


def test_row_maximum_scales_to_below_2_to_55():
    # the largest value of a row scales to an integer below 2^55 without rounding; the
    # top digit stays in [-128, 128] even when the lower digits borrow from it
    for a in (1.0 - 2.0 ** -53, -(1.0 - 2.0 ** -53), 0.75, 1.0 - 2.0 ** -20):
        X = to_int(a, exponent(abs(a)))
        assert abs(X) < 2 ** 55 and Fraction(X) == Fraction(a) * 2 ** (55 - exponent(abs(a)))
        d = digits(X)
        assert -128 <= d[0] <= 128
    assert digits(2 ** 55 - 4)[0] == 128


def test_levels_0_to_3_are_exact_in_fp32_over_256_terms():
    # the worst case: every digit at its extreme, all products of one sign
    L = [np.float32(0.0)] * 7
    exact = [0] * 7
    for _ in range(256):
        for s in range(7):
            for t in range(7 - s):
                prod = 128 * 128
                L[s + t] = np.float32(L[s + t] + np.float32(prod))
                exact[s + t] += prod
    for lvl in range(4):
        assert int(L[lvl]) == exact[lvl] and exact[lvl] <= 2 ** 24
    # level 4 may exceed 2^24 (then it can round): its weight is 2^-32 of level 0
    assert exact[4] > 2 ** 24


@pytest.mark.parametrize("nd", [7, 8])
@pytest.mark.parametrize("n,scale", [(300, 1.0), (700, 1e-8), (257, 3e5)])
def test_emulated_product_is_fp64_accurate(n, scale, nd):
    rng = np.random.default_rng(n)
    a = rng.standard_normal(n) * scale
    b = rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n))
    got, _, _ = emulate_dot(a, b, nd=nd)
    exact = sum(Fraction(x) * Fraction(y) for x, y in zip(a, b))
    # error class of an FP64 dot product, relative to the largest |a| |b| of the run
    bound = n * 2.0 ** -52 * np.abs(a).max() * np.abs(b).max()
    assert abs(Fraction(got) - exact) <= Fraction(bound)
    # and in practice near the FP64 rounding of the result itself
    assert abs(float(Fraction(got) - exact)) <= 64 * 2.0 ** -53 * float(abs(exact)) + \
        n ** 0.5 * 2.0 ** -55 * np.abs(a).max() * np.abs(b).max()


def test_integer_operands_give_exact_products():
    # small integers: every term is exact, so the product equals the exact sum
    rng = np.random.default_rng(3)
    a = rng.integers(-7, 8, 600).astype(np.float64)
    b = rng.integers(-5, 6, 600).astype(np.float64)
    got, _, _ = emulate_dot(a, b)
    assert got == float(np.dot(a.astype(np.int64), b.astype(np.int64)))


def test_dropping_a_digit_pair_breaks_fp64_accuracy():
    # planted mistake: the pairs with s + t = 6 left out (level 6 = 0)
    rng = np.random.default_rng(7)
    a, b = rng.standard_normal(300), rng.standard_normal(300)
    ea, eb = exponent(np.abs(a).max()), exponent(np.abs(b).max())
    da = [digits(to_int(x, ea)) for x in a]
    db = [digits(to_int(x, eb)) for x in b]
    L = [0] * 7
    for k in range(300):
        for s in range(7):
            for t in range(6 - s):       # s + t <= 5 only
                L[s + t] += da[k][s] * db[k][t]
    hi = (L[0] << 24) + (L[1] << 16) + (L[2] << 8) + L[3]
    lo = (L[4] << 16) + (L[5] << 8)
    got = math.ldexp(float(hi) * 16777216.0 + float(lo), ea + eb - 62)
    exact = float(sum(Fraction(x) * Fraction(y) for x, y in zip(a, b)))
    assert abs(got - exact) > 1e3 * 2.0 ** -53 * abs(exact)


def test_eight_digits_resolve_terms_far_below_the_row_maximum():
    # one large entry per row and many small ones (a localised orbital at a grid point):
    # seven digits resolve the small terms to 2^-55 of the maximum, eight to 2^-63
    rng = np.random.default_rng(11)
    a = rng.standard_normal(512) * 1e-3
    a[7] = 1.0
    b = rng.standard_normal(512)
    exact = sum(Fraction(x) * Fraction(y) for x, y in zip(a, b))
    err7 = abs(float(Fraction(emulate_dot(a, b, nd=7)[0]) - exact))
    err8 = abs(float(Fraction(emulate_dot(a, b, nd=8)[0]) - exact))
    assert err8 <= 2.0 ** -60 * 512 * np.abs(b).max()
    assert err8 < err7 / 16 or err7 == 0.0
