"""Host model of the split-precision energy epilogue's arithmetic (no GPU):
how much of the mixed-precision error the epilogue itself contributes.

The kernel receives W in FP32 (the tensor-core contractions' output) and
evaluates, per element orbit (the six orderings of one a < b < c) or per
element (orbits with repeated virtual indices):
  - the numerators sum_q Z_q W_q and sum_q Z_q Y_q in FP32 (Y from FP32 t1
    and ovov),
  - D = e_i + e_j + e_k - e_a - e_b - e_c in FP64,
  - 1/D as an FP32 reciprocal of the FP32 denominator refined by one
    Newton-Raphson step in FP64,
  - numerator x 1/D and all sums in FP64.
This file restates that arithmetic in numpy (float32 where the kernel uses
FP32) on the exact W of a task, and compares it with the same energy in FP64
throughout: the difference is the epilogue's share of the error, to be set
against the 1e-6 relative bound of the mixed-precision path (Sec. 4).  The
earlier all-FP32 scheme (FP32 denominators and FP32 sums) is modelled beside
it for comparison.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1609_08094_gb300 import synth
from tests.test_energy_forms import multiplicity, w_grouped, y_and_d


def recip64(d, r0):
    """One Newton-Raphson step for 1/d from the FP32 estimate r0."""
    r = np.float64(r0)
    return r + r * (1.0 - d * r)


def orbit_terms(w, y, eo, ev, i, j, k, f32_den, f32_sum):
    """E4, E5 of one task by element orbits, numerators in FP32.

    f32_den, f32_sum False: the kernel's scheme (FP64 denominator, Newton
    reciprocal, FP64 sums).  True: the earlier all-FP32 scheme (FP32
    denominator and reciprocal; terms summed in FP32 within each block orbit
    of 8^3 as a tree, and in FP64 across block orbits)."""
    f = np.float32
    v = len(ev)
    eijk = eo[i] + eo[j] + eo[k]
    w32, y32 = w.astype(f), y.astype(f)
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
        d64 = eijk - ev[a] - ev[b] - ev[c]
        if f32_den:
            r = f(1.0) / f(d64)
            t4, t5 = n4 * r, n5 * r
        else:
            r = recip64(d64, f(1.0) / f(d64))
            t4, t5 = np.float64(n4) * r, np.float64(n5) * r
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


def test_newton_reciprocal_is_fp64_accurate():
    rng = np.random.default_rng(3)
    d = -rng.uniform(1.2, 20.0, size=4000)
    r = recip64(d, (np.float32(1.0) / d.astype(np.float32)))
    assert np.max(np.abs(r * d - 1.0)) < 1e-13


@pytest.fixture(scope="module")
def inst():
    oracle.build()
    return synth.make_instance(3, 20, None, 31)


def test_epilogue_share_of_the_mixed_error(inst):
    """With the exact W, the kernel's epilogue arithmetic (FP32 numerators,
    FP64 denominators and sums) stays within 2e-8 of the FP64 energy of every
    task and within 1e-8 of the FP64 total; the earlier all-FP32 scheme is
    printed beside it."""
    rows = []
    tot_exact = np.zeros(2)
    tot_model = np.zeros(2)
    tot_f32 = np.zeros(2)
    for i, j, k in ((0, 1, 2), (0, 0, 1), (1, 2, 2), (0, 2, 2)):
        w = w_grouped(inst, i, j, k)
        y, d = y_and_d(inst, i, j, k)
        ex = np.array(exact_terms(w, y, d, i, j, k))
        mo = np.array(orbit_terms(w, y, inst.eps_occ, inst.eps_vir, i, j, k, False, False))
        ff = np.array(orbit_terms(w, y, inst.eps_occ, inst.eps_vir, i, j, k, True, True))
        tot_exact += ex
        tot_model += mo
        tot_f32 += ff
        rel_mo = abs(mo.sum() - ex.sum()) / abs(ex.sum())
        rel_ff = abs(ff.sum() - ex.sum()) / abs(ex.sum())
        rows.append((i, j, k, rel_mo, rel_ff))
        assert rel_mo <= 2e-8, (i, j, k, rel_mo)
    for r in rows:
        print("task (%d,%d,%d): epilogue model %.2e, all-FP32 scheme %.2e" % r)
    rel_tot = abs(tot_model.sum() - tot_exact.sum()) / abs(tot_exact.sum())
    rel_tot_f32 = abs(tot_f32.sum() - tot_exact.sum()) / abs(tot_exact.sum())
    print(f"total: epilogue model {rel_tot:.2e}, all-FP32 scheme {rel_tot_f32:.2e}")
    assert rel_tot <= 1e-8
