"""Host model of the split-precision energy epilogue's arithmetic (no GPU):
how much of the mixed-precision error the epilogue itself contributes.

The kernel receives W in FP32 (the tensor-core contractions' output) and
evaluates, per element orbit (the six orderings of one a < b < c) or per
element (orbits with repeated virtual indices):
  - the numerators sum_q Z_q W_q and sum_q Z_q Y_q in FP32 (Y from FP32 t1
    and ovov),
  - D = e_i + e_j + e_k - e_a - e_b - e_c, 1/D and numerator x 1/D in
    float-float (double-FP32) arithmetic: TwoSum / Fast2Sum for the sums,
    an FP32 reciprocal corrected with the exact FMA residual, the exact FMA
    error of the product,
  - the terms summed in float-float per thread and over the CTA, then in
    FP64 over the task (the float-float sums are modelled as FP64 sums:
    their error, ~1e-12 relative, is far below the rest).
This file restates that arithmetic in numpy (float32 where the kernel uses
FP32; an FMA as the float64 product and sum rounded once to float32) on the
exact W of a task, and compares it with the same energy in FP64 throughout:
the difference is the epilogue's share of the error, to be set against the
1e-6 relative bound of the mixed-precision path (Sec. 4).  Two cheaper
schemes are modelled beside it for comparison: FP32 denominators with FP64
sums, and FP32 denominators with FP32 sums within each 8^3 block orbit.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1609_08094_gb300 import synth
from tests.test_energy_forms import multiplicity, w_grouped, y_and_d


F32 = np.float32


def fmaf(a, b, c):
    """a * b + c rounded once to float32 (the float64 product of two floats is exact)."""
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


def ff_of(x):
    hi = F32(x)
    return hi, F32(np.float64(x) - np.float64(hi))


def ff_two_sum(a, b):
    s = F32(a + b)
    bb = F32(s - a)
    return s, F32(F32(a - F32(s - bb)) + F32(b - bb))


def ff_fast(a, b):
    s = F32(a + b)
    return s, F32(b - F32(s - a))


def ff_sub(a, b):
    s, e = ff_two_sum(a[0], F32(-b[0]))
    return ff_fast(s, F32(e + F32(a[1] - b[1])))


def ff_recip(d):
    r = F32(F32(1.0) / d[0])
    e = fmaf(-d[1], r, fmaf(-d[0], r, F32(1.0)))
    return r, F32(r * e)


def ff_mul(x, r):
    p = F32(x * r[0])
    return ff_fast(p, fmaf(x, r[1], fmaf(x, r[0], -p)))


def ff_value(a):
    return np.float64(a[0]) + np.float64(a[1])


def orbit_terms(w, y, eo, ev, i, j, k, f32_den, f32_sum):
    """E4, E5 of one task by element orbits, numerators in FP32.

    f32_den False: the kernel's scheme (float-float denominator, reciprocal
    and product; FP64 sums).  f32_den True: FP32 denominator, reciprocal and
    product, with FP64 sums (f32_sum False) or FP32 sums within each block
    orbit of 8^3 as a tree and FP64 across block orbits (f32_sum True)."""
    f = np.float32
    v = len(ev)
    eijk = eo[i] + eo[j] + eo[k]
    w32, y32 = w.astype(f), y.astype(f)
    ev_ff = [ff_of(x) for x in ev]
    eijk_ff = ff_of(eijk)
    per_orbit = {}
    for a, b, c in itertools.product(range(v), repeat=3):
        if a < b < c:
            order = [(a, b, c), (a, c, b), (b, a, c), (b, c, a), (c, a, b), (c, b, a)]
            ws = [w32[x] for x in order]
            ys = [y32[x] for x in order]
            E = ws[0] + ws[3] + ws[4]
            O = ws[1] + ws[2] + ws[5]
            ww = f(0.0)
            wy = f(0.0)
            for q in range(6):
                ww = ww + ws[q] * ws[q]
                wy = wy + ws[q] * ys[q]
            n4 = f(6) * ww + f(2) * (E * E + O * O) - f(8) * E * O
            n5 = f(6) * wy + (f(2) * E - f(4) * O) * (ys[0] + ys[3] + ys[4]) \
                + (f(2) * O - f(4) * E) * (ys[1] + ys[2] + ys[5])
        elif len({a, b, c}) < 3:
            x = (a, b, c)
            z = f(8) * w32[x] - f(4) * (w32[a, c, b] + w32[b, a, c] + w32[c, b, a]) \
                + f(2) * (w32[b, c, a] + w32[c, a, b])
            n4 = z * w32[x]
            n5 = z * y32[x]
        else:
            continue
        if f32_den:
            r = f(1.0) / f(eijk - ev[a] - ev[b] - ev[c])
            t4, t5 = n4 * r, n5 * r
        else:
            dd = ff_sub(ff_sub(ff_sub(eijk_ff, ev_ff[a]), ev_ff[b]), ev_ff[c])
            r = ff_recip(dd)
            t4, t5 = ff_value(ff_mul(n4, r)), ff_value(ff_mul(n5, r))
        key = tuple(sorted((a // 8, b // 8, c // 8)))
        per_orbit.setdefault(key, []).append((t4, t5))
    e4 = e5 = 0.0
    for terms in per_orbit.values():
        arr = np.array(terms, dtype=np.float32 if f32_sum else np.float64)
        s = arr.sum(axis=0)  # pairwise: a tree like the kernel's shuffles
        e4 += float(s[0])
        e5 += float(s[1])
    m = multiplicity(i, j, k)
    return m / 6 * e4, m / 6 * e5


def exact_terms(w, y, d, i, j, k):
    from tests.test_energy_forms import z_of
    z = z_of(w)
    m = multiplicity(i, j, k)
    return m / 6 * float(np.sum(z * w / d)), m / 6 * float(np.sum(z * y / d))


def test_float_float_quotient_is_fp64_accurate():
    """x / D in float-float, with D formed by float-float subtractions from
    energies rounded to ~48 bits: within 2e-13 of the FP64 quotient."""
    rng = np.random.default_rng(3)
    worst = 0.0
    for _ in range(3000):
        eo = -rng.uniform(0.3, 2.0, size=3)
        ev = rng.uniform(0.1, 5.0, size=3)
        x = F32(rng.normal() * 10.0 ** rng.uniform(-6, 2))
        d = ff_sub(ff_sub(ff_sub(ff_of(eo.sum()), ff_of(ev[0])), ff_of(ev[1])), ff_of(ev[2]))
        got = ff_value(ff_mul(x, ff_recip(d)))
        ref = np.float64(x) / (eo.sum() - ev[0] - ev[1] - ev[2])
        worst = max(worst, abs(got - ref) / abs(ref))
    assert worst < 2e-13, worst


@pytest.fixture(scope="module")
def inst():
    oracle.build()
    return synth.make_instance(3, 20, None, 31)


def test_epilogue_share_of_the_mixed_error(inst):
    """With the exact W, the kernel's epilogue arithmetic (FP32 numerators,
    float-float denominators and products, FP64 sums) stays within 2e-8 of
    the FP64 energy of every task and within 1e-8 of the FP64 total; the
    two cheaper schemes are printed beside it."""
    rows = []
    tot_exact = np.zeros(2)
    tot_model = np.zeros(2)
    tot_f32 = np.zeros(2)
    for i, j, k in ((0, 1, 2), (0, 0, 1), (1, 2, 2), (0, 2, 2)):
        w = w_grouped(inst, i, j, k)
        y, d = y_and_d(inst, i, j, k)
        ex = np.array(exact_terms(w, y, d, i, j, k))
        mo = np.array(orbit_terms(w, y, inst.eps_occ, inst.eps_vir, i, j, k, False, False))
        fd = np.array(orbit_terms(w, y, inst.eps_occ, inst.eps_vir, i, j, k, True, False))
        ff = np.array(orbit_terms(w, y, inst.eps_occ, inst.eps_vir, i, j, k, True, True))
        tot_exact += ex
        tot_model += mo
        tot_f32 += ff
        rel_mo = abs(mo.sum() - ex.sum()) / abs(ex.sum())
        rel_fd = abs(fd.sum() - ex.sum()) / abs(ex.sum())
        rel_ff = abs(ff.sum() - ex.sum()) / abs(ex.sum())
        rows.append((i, j, k, rel_mo, rel_fd, rel_ff))
        assert rel_mo <= 2e-8, (i, j, k, rel_mo)
    for r in rows:
        print("task (%d,%d,%d): epilogue model %.2e, FP32 denominators %.2e, all-FP32 %.2e" % r)
    rel_tot = abs(tot_model.sum() - tot_exact.sum()) / abs(tot_exact.sum())
    rel_tot_f32 = abs(tot_f32.sum() - tot_exact.sum()) / abs(tot_exact.sum())
    print(f"total: epilogue model {rel_tot:.2e}, all-FP32 scheme {rel_tot_f32:.2e}")
    assert rel_tot <= 1e-8
