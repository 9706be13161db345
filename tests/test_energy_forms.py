"""The algebraic forms the CUDA kernels evaluate, restated in numpy on the
host (no GPU) and checked against the oracle, which uses none of them:

1. W of a task as three grouped contractions, one per "single" virtual index
   (s; p, q) in {(i; j, k), (j; i, k), (k; i, j)}, each a GEMM over the K
   segments [d | d | l | l] (the six permutations of Eq. symm_operator
   applied to Eq. analytical_triples_ampl, grouped):
     U^{s;p,q}[a][b][c] = sum_d t^{ad}_{sp} (db|cq) + sum_d t^{ad}_{sq} (dc|bp)
                        - sum_l (as|lq) t^{bc}_{pl} - sum_l (as|lp) t^{cb}_{ql}
     W^{abc} = U^{i;j,k}[a][b][c] + U^{j;i,k}[b][a][c] + U^{k;i,j}[c][a][b]
2. The task energy in the Z form of the restricted loop (Sec. 3): with m the
   number of distinct orderings of (i, j, k),
     e_ijk = (m/6) sum_abc Z (W + Y) / D,
     Z = 8 W - 4 (W_acb + W_bac + W_cba) + 2 (W_bca + W_cab).
3. The element-orbit expansion of 2 used for the orbits of three distinct
   virtual indices: over the six orderings q of one (a, b, c), with E and O
   the sums of W over the even and odd orderings,
     sum_q Z_q W_q = 6 sum w^2 + 2 E^2 + 2 O^2 - 8 E O,
     sum_q Z_q Y_q = 6 sum w y + (2E - 4O)(y_even) + (2O - 4E)(y_odd).
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1609_08094_gb300 import synth


def u_group(inst, s, p, q):
    """U^{s;p,q}[a][b][c] by the four K segments."""
    t2, vvvo, ooov = inst.t2, inst.vvvo, inst.ooov
    # (db|cq) = vvvo[d][b][c][q]; (dc|bp) = vvvo[d][c][b][p]
    # (as|lq) = (ql|sa) = ooov[q][l][s][a]
    u = np.einsum("ad,dbc->abc", t2[s, p], vvvo[:, :, :, q])
    u += np.einsum("ad,dcb->abc", t2[s, q], vvvo[:, :, :, p])
    u -= np.einsum("la,lbc->abc", ooov[q, :, s, :], t2[p])
    u -= np.einsum("la,lcb->abc", ooov[p, :, s, :], t2[q])
    return u


def w_grouped(inst, i, j, k):
    return (u_group(inst, i, j, k)
            + u_group(inst, j, i, k).transpose(1, 0, 2)
            + u_group(inst, k, i, j).transpose(1, 2, 0))


def y_and_d(inst, i, j, k):
    t1, ov, eo, ev = inst.t1, inst.ovov, inst.eps_occ, inst.eps_vir
    y = (np.einsum("a,bc->abc", t1[i], ov[j, :, k, :]) + np.einsum("b,ac->abc", t1[j], ov[i, :, k, :])
         + np.einsum("c,ab->abc", t1[k], ov[i, :, j, :]))
    d = eo[i] + eo[j] + eo[k] - ev[:, None, None] - ev[None, :, None] - ev[None, None, :]
    return y, d


def z_of(w):
    return (8 * w - 4 * (w.transpose(0, 2, 1) + w.transpose(1, 0, 2) + w.transpose(2, 1, 0))
            + 2 * (w.transpose(1, 2, 0) + w.transpose(2, 0, 1)))


def multiplicity(i, j, k):
    return len(set(itertools.permutations((i, j, k))))


def z_form(inst, i, j, k):
    w = w_grouped(inst, i, j, k)
    y, d = y_and_d(inst, i, j, k)
    z, m = z_of(w), multiplicity(i, j, k)
    return m / 6 * np.sum(z * w / d), m / 6 * np.sum(z * y / d)


def element_orbit_form(inst, i, j, k):
    """Distinct a < b < c by the E/O expansion, every other (a, b, c) by the
    Z form element by element."""
    w = w_grouped(inst, i, j, k)
    y, d = y_and_d(inst, i, j, k)
    z, m, v = z_of(w), multiplicity(i, j, k), inst.v
    e4 = e5 = 0.0
    for a, b, c in itertools.product(range(v), repeat=3):
        if a < b < c:
            order = [(a, b, c), (a, c, b), (b, a, c), (b, c, a), (c, a, b), (c, b, a)]
            ws = [w[x] for x in order]
            ys = [y[x] for x in order]
            ev_, od = ws[0] + ws[3] + ws[4], ws[1] + ws[2] + ws[5]
            s4 = 6 * sum(x * x for x in ws) + 2 * ev_ ** 2 + 2 * od ** 2 - 8 * ev_ * od
            s5 = (6 * sum(x * yy for x, yy in zip(ws, ys)) + (2 * ev_ - 4 * od) * (ys[0] + ys[3] + ys[4])
                  + (2 * od - 4 * ev_) * (ys[1] + ys[2] + ys[5]))
            e4 += s4 / d[a, b, c]
            e5 += s5 / d[a, b, c]
        elif len({a, b, c}) < 3:
            e4 += z[a, b, c] * w[a, b, c] / d[a, b, c]
            e5 += z[a, b, c] * y[a, b, c] / d[a, b, c]
    return m / 6 * e4, m / 6 * e5


@pytest.fixture(scope="module")
def inst():
    oracle.build()
    return synth.make_instance(4, 7, None, 21)


def test_grouped_contractions_and_z_form_equal_the_oracle(inst):
    tasks = oracle.sorted_triples(inst.o)
    ref = oracle.triple_energies(inst, tasks)
    scale = np.abs(ref).max()
    for n, (i, j, k) in enumerate(tasks):
        e4, e5 = z_form(inst, int(i), int(j), int(k))
        assert abs(e4 - ref[n, 0]) <= 1e-12 * scale, (i, j, k)
        assert abs(e5 - ref[n, 1]) <= 1e-12 * scale, (i, j, k)


def test_element_orbit_expansion_equals_the_z_form(inst):
    scale = abs(z_form(inst, 0, 1, 2)[0])  # i = j = k is an exact zero: one absolute scale
    for i, j, k in ((0, 1, 2), (0, 0, 3), (1, 2, 2), (1, 1, 1)):
        z4, z5 = z_form(inst, i, j, k)
        o4, o5 = element_orbit_form(inst, i, j, k)
        assert abs(o4 - z4) <= 1e-12 * scale
        assert abs(o5 - z5) <= 1e-12 * scale


def test_e4_quadratic_form_is_nonnegative():
    """6 sum w^2 + 2E^2 + 2O^2 - 8EO >= 0 for any six values: with the
    denominators negative this keeps every element orbit's E[4] term <= 0."""
    rng = np.random.default_rng(5)
    for _ in range(2000):
        ws = rng.normal(size=6) * rng.choice([1e-3, 1.0, 1e3])
        ev_, od = ws[0] + ws[3] + ws[4], ws[1] + ws[2] + ws[5]
        q = 6 * np.sum(ws * ws) + 2 * ev_ ** 2 + 2 * od ** 2 - 8 * ev_ * od
        assert q >= -1e-12 * 6 * np.sum(ws * ws)
