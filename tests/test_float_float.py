"""Host model of the float-float arithmetic of the FP64-emulation path (no GPU).

The FP64 emulation stores U as (hi, lo) FP32 pairs formed from its exact int64
totals (int64_to_ff in gemm_oz.cu) and runs the energy epilogue in float-float
arithmetic (the dd type in epilogue.cu): sums by TwoSum + Fast2Sum, products
from the FMA residual of hi x hi plus the cross terms, quotients through an
FP32 reciprocal with one Newton correction.  These tests restate those steps
in numpy float32 (an FMA as the exact float64 product plus the addend, rounded
once) and bound their relative error against exact rationals: well below the
1e-10 tolerance of the FP64-emulation path (Sec. 4 asks FP64 accuracy of it).
"""
from fractions import Fraction

import numpy as np
import pytest

F32 = np.float32


def fmaf(a, b, c):
    return F32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def two_sum(a, b):
    s = F32(a + b)
    bb = F32(s - a)
    return s, F32(F32(a - F32(s - bb)) + F32(b - bb))


def fast(a, b):
    s = F32(a + b)
    return s, F32(b - F32(s - a))


def dd_add(a, b):
    s, e = two_sum(a[0], b[0])
    return fast(s, F32(e + F32(a[1] + b[1])))


def dd_mul(a, b):
    p = F32(a[0] * b[0])
    e = fmaf(a[0], b[0], -p)
    e = fmaf(a[0], b[1], fmaf(a[1], b[0], e))
    return fast(p, e)


def dd_recip(d):
    r = F32(F32(1.0) / d[0])
    e = fmaf(-d[1], r, fmaf(-d[0], r, F32(1.0)))
    return r, F32(r * e)


def int64_to_ff(t, k):
    t2 = t >> 48
    rem = t - (t2 << 48)
    f2 = F32(t2) * F32(2.0 ** 48)
    f1 = F32(rem >> 24) * F32(2.0 ** 24)
    f0 = F32(rem & 0xFFFFFF)
    s = F32(f2 + f1)
    bb = F32(s - f2)
    e = F32(F32(f2 - F32(s - bb)) + F32(f1 - bb))
    s2 = F32(s + f0)
    b2 = F32(s2 - s)
    e = F32(e + F32(F32(s - F32(s2 - b2)) + F32(f0 - b2)))
    hi = F32(s2 + e)
    lo = F32(e - F32(hi - s2))
    return F32(np.ldexp(hi, k)), F32(np.ldexp(lo, k))


def value(p):
    return Fraction(float(p[0])) + Fraction(float(p[1]))


def dd_of(x):
    hi = F32(x)
    return hi, F32(x - float(hi))


def test_int64_totals_become_pairs_to_48_bits():
    rng = np.random.default_rng(11)
    ts = [0, 1, -1, (1 << 24) - 1, -(1 << 40) + 12345, (1 << 55) + 987654321, -(1 << 62) + 3]
    ts += [int(x) for x in rng.integers(-(1 << 62), 1 << 62, size=400)]
    ts += [int(x) for x in rng.integers(-(1 << 30), 1 << 30, size=100)]
    for t in ts:
        for k in (-60, -42, 0):
            got = value(int64_to_ff(t, k))
            exact = Fraction(t) * Fraction(2) ** k
            if t == 0:
                assert got == 0
                continue
            assert abs(got - exact) <= abs(exact) * Fraction(1, 2 ** 46), (t, k)
            if abs(t) < (1 << 24):
                assert got == exact  # one part: exact


def test_dd_operations_are_fp64_accurate():
    rng = np.random.default_rng(12)
    xs = rng.standard_normal(300) * 10.0 ** rng.uniform(-4, 3, 300)
    ys = rng.standard_normal(300) * 10.0 ** rng.uniform(-4, 3, 300)
    worst = {"add": 0.0, "mul": 0.0, "div": 0.0}
    for x, y in zip(xs, ys):
        a, b = dd_of(x), dd_of(y)
        ea, eb = value(a), value(b)
        s = value(dd_add(a, b))
        worst["add"] = max(worst["add"], float(abs(s - (ea + eb)) / (abs(ea) + abs(eb))))
        m = value(dd_mul(a, b))
        worst["mul"] = max(worst["mul"], float(abs(m - ea * eb) / abs(ea * eb)))
        q = value(dd_mul(a, dd_recip(b)))
        worst["div"] = max(worst["div"], float(abs(q - ea / eb) / abs(ea / eb)))
    print(worst)
    assert worst["add"] <= 2.0 ** -44
    assert worst["mul"] <= 2.0 ** -44
    assert worst["div"] <= 2.0 ** -42
