"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(no GPU).  Each pin is chosen so that a plausible slip in the oracle -- a
dropped term of P, a wrong sign of the denominator, a transposed amplitude or
integral, a wrong tilde constant -- fails at least one of them; the mutation
test at the end checks that claim on a deliberately broken copy of the
equations."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1609_08094_gb300 import synth
from tests import spin_orbital

SIZES = [(2, 3), (3, 3), (2, 4), (3, 4), (4, 5), (3, 7), (4, 20)]


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("o,v", SIZES)
def test_oracle_equals_bruteforce(oracle_lib, o, v):
    inst = synth.make_instance(o, v, seed=100 + o * 31 + v)
    e = oracle.energy(inst)
    b = oracle.bruteforce(inst)
    for x, y in zip(e, b):
        assert rel(x, y) < 1e-13


@pytest.mark.parametrize("o,v", [(2, 3), (3, 4), (4, 6)])
def test_task_shares_equal_bruteforce_orderings(oracle_lib, o, v):
    """Each sorted-triple task equals the brute-force summands of its distinct
    orderings (the restricted loop of Sec. 3 loses nothing)."""
    inst = synth.make_instance(o, v, seed=5)
    tasks = oracle.sorted_triples(o)
    e = oracle.triple_energies(inst, tasks)
    f4, f5 = oracle.bruteforce(inst, per_triple=True)
    for t, (i, j, k) in enumerate(tasks):
        orders = set(itertools.permutations((int(i), int(j), int(k))))
        s4 = sum(f4[p] for p in orders)
        s5 = sum(f5[p] for p in orders)
        scale = np.abs(f4).max() + np.abs(f5).max()
        assert abs(e[t, 0] - s4) <= 1e-13 * scale
        assert abs(e[t, 1] - s5) <= 1e-13 * scale


@pytest.mark.parametrize("o,v", [(2, 3), (3, 3), (2, 4), (3, 4), (4, 4)])
def test_oracle_equals_spin_orbital_textbook(oracle_lib, o, v):
    """Strongest pin: the spin-orbital (T) formula on the spin-expanded inputs
    (independent of the paper's spatial equations and of their sign)."""
    inst = synth.make_instance(o, v, seed=17 * o + v)
    e4, e5, e = oracle.energy(inst)
    es, es4 = spin_orbital.energy(inst)
    assert rel(e, es) < 1e-12
    assert rel(e4, es4) < 1e-12


def test_zero_when_single_occupied_or_virtual(oracle_lib):
    for o, v in [(1, 1), (1, 5), (1, 12), (3, 1), (5, 1)]:
        inst = synth.make_instance(o, v, seed=3)
        e = oracle.energy(inst)
        *_, scale = oracle.bruteforce(inst, with_scale=True)
        assert abs(e[2]) <= 1e-12 * max(scale, 1e-300) + 1e-300


def test_zero_amplitudes_give_zero(oracle_lib):
    inst = synth.make_instance(3, 5, seed=4)
    inst.t1 = np.zeros_like(inst.t1)
    inst.t2 = np.zeros_like(inst.t2)
    assert oracle.energy(inst) == (0.0, 0.0, 0.0)


def test_zero_singles_give_zero_e5(oracle_lib):
    inst = synth.make_instance(3, 6, seed=8)
    inst.t1 = np.zeros_like(inst.t1)
    e4, e5, e = oracle.energy(inst)
    assert e5 == 0.0 and e == e4 and e4 < 0


def test_diagonal_triples_vanish(oracle_lib):
    inst = synth.make_instance(4, 9, seed=9)
    diag = np.array([[i, i, i] for i in range(4)], dtype=np.int32)
    e = oracle.triple_energies(inst, diag)
    scale = np.abs(oracle.triple_energies(inst, oracle.sorted_triples(4))).max()
    assert np.all(np.abs(e) <= 1e-13 * scale)


def test_e4_nonpositive_per_task(oracle_lib):
    for o, v in [(3, 5), (4, 20), (5, 8)]:
        inst = synth.make_instance(o, v, seed=o + v)
        e = oracle.triple_energies(inst, oracle.sorted_triples(o))
        scale = np.abs(e[:, 0]).max()
        assert np.all(e[:, 0] <= 1e-13 * scale)


def test_quartic_scaling(oracle_lib):
    """Integrals, T1 and T2 all times s => every energy times s^4."""
    inst = synth.make_instance(3, 6, seed=12)
    base = oracle.energy(inst)
    s = 1.7
    for name in ("t1", "t2", "vvvo", "ooov", "ovov"):
        setattr(inst, name, getattr(inst, name) * s)
    scaled = oracle.energy(inst)
    for x, y in zip(scaled, base):
        assert rel(x, y * s ** 4) < 1e-13


def test_e5_linear_in_singles(oracle_lib):
    inst = synth.make_instance(3, 6, seed=13)
    e4, e5, _ = oracle.energy(inst)
    inst.t1 = inst.t1 * -2.5
    f4, f5, _ = oracle.energy(inst)
    assert rel(f4, e4) < 1e-14
    assert rel(f5, -2.5 * e5) < 1e-13


def _relabel(inst, perm_o=None, perm_v=None):
    o, v = inst.o, inst.v
    po = np.arange(o) if perm_o is None else np.asarray(perm_o)
    pv = np.arange(v) if perm_v is None else np.asarray(perm_v)
    out = synth.Instance(o, v, inst.naux, inst.seed,
                         inst.eps_occ[po], inst.eps_vir[pv],
                         inst.t1[np.ix_(po, pv)],
                         inst.t2[np.ix_(po, po, pv, pv)],
                         inst.vvvo[np.ix_(pv, pv, pv, po)],
                         inst.ooov[np.ix_(po, po, po, pv)],
                         inst.ovov[np.ix_(po, pv, po, pv)])
    return out


def test_relabelling_invariance(oracle_lib):
    inst = synth.make_instance(4, 7, seed=21)
    base = oracle.energy(inst)
    rng = np.random.default_rng(0)
    for kind in ("occ", "vir", "both"):
        po = rng.permutation(4) if kind in ("occ", "both") else None
        pv = rng.permutation(7) if kind in ("vir", "both") else None
        e = oracle.energy(_relabel(inst, po, pv))
        for x, y in zip(e, base):
            assert rel(x, y) < 1e-13


def _mutated_energy(inst, mutation):
    """The paper's equations with one planted mistake (test-local copy)."""
    eo, ev, t1, t2 = inst.eps_occ, inst.eps_vir, inst.t1, inst.t2
    vvvo, ooov, ovov = inst.vvvo, inst.ooov, inst.ovov
    if mutation == "transposed_t2":
        t2 = t2.transpose(0, 1, 3, 2)
    vv = "ijad,bdck->ijkabc" if mutation != "wrong_integral_index" else "ijad,cdbk->ijkabc"
    X = np.einsum(vv, t2, vvvo) - np.einsum("ilab,ljkc->ijkabc", t2, ooov)
    if mutation == "wrong_sign_ooov":
        X = np.einsum(vv, t2, vvvo) + np.einsum("ilab,ljkc->ijkabc", t2, ooov)
    terms = ["ijkabc", "ikjacb", "jikbac", "jkibca", "kijcab", "kjicba"]
    if mutation == "dropped_P_term":
        terms = terms[:-1]
    W = sum(np.einsum(t + "->ijkabc", X) for t in terms)
    Y = (np.einsum("ia,jbkc->ijkabc", t1, ovov) + np.einsum("jb,iakc->ijkabc", t1, ovov)
         + np.einsum("kc,iajb->ijkabc", t1, ovov))
    D = (eo[:, None, None, None, None, None] + eo[None, :, None, None, None, None]
         + eo[None, None, :, None, None, None] - ev[None, None, None, :, None, None]
         - ev[None, None, None, None, :, None] - ev[None, None, None, None, None, :])
    if mutation == "literal_paper_sign":
        D = -D
    c3 = 1.0 / 3.0 if mutation == "wrong_tilde_constant" else 2.0 / 3.0

    def tilde(x):
        return (4.0 / 3.0 * x - 2.0 * np.einsum("ijkacb->ijkabc", x)
                + c3 * np.einsum("ijkbca->ijkabc", x))
    return float(np.sum(tilde(W) * (W + Y) / D) if mutation != "e5_without_tilde"
                 else np.sum(tilde(W) * W / D) + np.sum(Y * W / D))


@pytest.mark.parametrize("mutation", ["none", "transposed_t2", "wrong_integral_index",
                                      "wrong_sign_ooov", "dropped_P_term",
                                      "literal_paper_sign", "wrong_tilde_constant",
                                      "e5_without_tilde"])
def test_pins_catch_planted_mistakes(oracle_lib, mutation):
    inst = synth.make_instance(3, 4, seed=77)
    es, _ = spin_orbital.energy(inst)
    em = _mutated_energy(inst, mutation)
    if mutation == "none":
        assert rel(em, es) < 1e-12
    else:
        assert rel(em, es) > 1e-6, mutation
