"""Pins of the RI-MP2 oracle (Sec. 2.1) against facts independent of it:

* the spin-orbital textbook MP2 energy, 1/4 sum_IJAB |<IJ||AB>|^2 / (f_I + f_J
  - f_A - f_B) (Szabo & Ostlund eq. 6.74), built from the same ERIs expanded to
  spin orbitals;
* the MP2 energy of the same synthetic system written with its MP1 doubles
  amplitudes and its (ia|jb) block (an independent product path through the
  (T) generator): E = sum t^ab_ij [2 (ia|jb) - (ib|ja)];
* E <= 0 (for each pair and each (a, b), 2(x^2 + y^2) - 2xy >= 0 with a
  symmetric positive denominator), E(sC) = s^4 E(C), C = 0 => E = 0, and
  invariance under relabelling occupied and virtual orbitals;
* a planted mistake (the exchange term with g_ab instead of g_ba, a dropped
  factor 2) fails the textbook pin."""
import numpy as np
import pytest

import oracle
from paper_1609_08094_gb300 import synth


def textbook_mp2(inst):
    o, v = inst.o, inst.v
    C = np.asarray(inst.C)
    g = np.einsum("qai,qbj->iajb", C, C)                 # (ia|jb)
    O, V = 2 * o, 2 * v
    io, iv = np.arange(O) // 2, np.arange(V) // 2
    so, sv = np.arange(O) % 2, np.arange(V) % 2
    dov = (so[:, None] == sv[None, :]).astype(np.float64)
    # <IJ|AB> = (IA|JB) delta(s_I,s_A) delta(s_J,s_B)
    gs = g[io][:, iv][:, :, io][:, :, :, iv]             # [I][A][J][B]
    ijab = gs.transpose(0, 2, 1, 3) * dov[:, None, :, None] * dov[None, :, None, :]
    anti = ijab - ijab.transpose(0, 1, 3, 2)
    eo, ev = np.asarray(inst.eps_occ)[io], np.asarray(inst.eps_vir)[iv]
    den = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    return 0.25 * float(np.sum(anti * anti / den))


@pytest.mark.parametrize("o,v,naux,seed", [(2, 3, 5, 1), (3, 5, 7, 2), (4, 6, None, 3), (1, 4, 3, 4)])
def test_oracle_equals_spin_orbital_textbook(o, v, naux, seed):
    inst = synth.make_mp2_instance(o, v, naux, seed)
    e = oracle.mp2_energy(inst)[2]
    ref = textbook_mp2(inst)
    assert e == pytest.approx(ref, rel=1e-12, abs=1e-15)
    assert e < 0


def test_oracle_equals_mp1_amplitude_form():
    o, v, naux, seed = 4, 9, None, 5
    t = synth.make_instance(o, v, naux, seed)          # same system: t2 = (ia|jb)/(e_i+e_j-e_a-e_b)
    m = synth.make_mp2_instance(o, v, naux, seed)
    g = np.asarray(t.ovov)                              # [i][a][j][b]
    t2 = np.asarray(t.t2)                               # [i][j][a][b]
    gij = g.transpose(0, 2, 1, 3)                       # [i][j][a][b] = (ia|jb)
    e_ref = float(np.sum(t2 * (2.0 * gij - gij.transpose(0, 1, 3, 2))))
    assert oracle.mp2_energy(m)[2] == pytest.approx(e_ref, rel=1e-12)


def test_exact_zero_scaling_and_sign():
    inst = synth.make_mp2_instance(3, 7, 10, 6)
    ej, ek, e = oracle.mp2_energy(inst)
    assert e < 0 and ej < 0 and e == pytest.approx(ej + ek)
    s = 1.7
    sc = synth.Mp2Instance(inst.o, inst.v, inst.naux, inst.seed, inst.eps_occ, inst.eps_vir,
                           np.asarray(inst.C) * s)
    assert oracle.mp2_energy(sc)[2] == pytest.approx(s ** 4 * e, rel=1e-12)
    zero = synth.Mp2Instance(inst.o, inst.v, inst.naux, inst.seed, inst.eps_occ, inst.eps_vir,
                             np.zeros_like(inst.C))
    assert oracle.mp2_energy(zero) == (0.0, 0.0, 0.0)


def test_relabelling_invariance():
    inst = synth.make_mp2_instance(4, 8, 11, 7)
    e = oracle.mp2_energy(inst)[2]
    rng = np.random.default_rng(0)
    po, pv = rng.permutation(4), rng.permutation(8)
    C = np.asarray(inst.C)[:, pv][:, :, po]
    perm = synth.Mp2Instance(4, 8, 11, 7, np.asarray(inst.eps_occ)[po], np.asarray(inst.eps_vir)[pv], C)
    assert oracle.mp2_energy(perm)[2] == pytest.approx(e, rel=1e-13)


@pytest.mark.parametrize("mistake", ["exchange_untransposed", "no_factor_two"])
def test_planted_mistakes_fail_the_textbook_pin(mistake):
    inst = synth.make_mp2_instance(3, 5, 7, 8)
    C = np.asarray(inst.C)
    eo, ev = np.asarray(inst.eps_occ), np.asarray(inst.eps_vir)
    e = 0.0
    for i in range(3):
        for j in range(3):
            g = C[:, :, i].T @ C[:, :, j]
            eps = ev[:, None] + ev[None, :] - eo[i] - eo[j]
            x = g if mistake == "exchange_untransposed" else g.T
            f = 2.0 if mistake == "exchange_untransposed" else 1.0
            e -= float(np.sum(g * (f * g - x) / eps))
    assert abs(e - textbook_mp2(inst)) > 1e-6 * abs(textbook_mp2(inst))


def test_pair_restricted_loop_equals_full_loop():
    """The restricted i <= j loop (Eq. tasks_rimp2: o(o+1)/2 pair tasks),
    with weight 2 off the diagonal, equals the full ordered-pair sum."""
    inst = synth.make_mp2_instance(5, 6, 9, 9)
    C = np.asarray(inst.C)
    eo, ev = np.asarray(inst.eps_occ), np.asarray(inst.eps_vir)
    e = 0.0
    for i in range(5):
        for j in range(i, 5):
            g = C[:, :, i].T @ C[:, :, j]
            eps = ev[:, None] + ev[None, :] - eo[i] - eo[j]
            e -= (1.0 if i == j else 2.0) * float(np.sum(g * (2 * g - g.T) / eps))
    assert e == pytest.approx(oracle.mp2_energy(inst)[2], rel=1e-13)
