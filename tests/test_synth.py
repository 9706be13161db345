"""The seeded input generator: distributions, symmetries and the MP1 relation
(no GPU)."""
import numpy as np

from paper_1609_08094_gb300 import synth


def test_uniform_counter_based_and_reproducible():
    a = synth.uniform(5, 1, 1000)
    b = synth.uniform(5, 1, 600, offset=400)
    assert np.array_equal(a[400:], b)
    assert a.min() >= 0.0 and a.max() < 1.0
    assert not np.array_equal(a, synth.uniform(6, 1, 1000))
    assert not np.array_equal(a, synth.uniform(5, 2, 1000))


def test_normal_moments():
    z = synth.normal(3, 1, 400000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_integral_symmetry_and_blocks():
    inst = synth.make_instance(3, 5, seed=2)
    o, v = 3, 5
    assert np.allclose(inst.ovov, inst.ovov.transpose(2, 3, 0, 1), rtol=0, atol=1e-15)
    assert np.allclose(inst.vvvo, inst.vvvo.transpose(1, 0, 2, 3), rtol=0, atol=1e-15)
    assert np.allclose(inst.ooov, inst.ooov.transpose(1, 0, 2, 3), rtol=0, atol=1e-15)
    B = synth.factors(o, v, inst.naux, 2)
    assert np.array_equal(B, B.transpose(0, 2, 1))
    # (pq|rs) = sum_Q B^Q_pq B^Q_rs, spot checks in every block
    full = np.einsum("Qpq,Qrs->pqrs", B, B)
    assert np.allclose(inst.vvvo, full[o:, o:, o:, :o], atol=1e-14)
    assert np.allclose(inst.ooov, full[:o, :o, :o, o:], atol=1e-14)
    assert np.allclose(inst.ovov, full[:o, o:, :o, o:], atol=1e-14)


def test_mp1_doubles_and_ranges():
    inst = synth.make_instance(4, 9, seed=11)
    eo, ev = inst.eps_occ, inst.eps_vir
    D = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    assert np.allclose(inst.t2 * D, inst.ovov.transpose(0, 2, 1, 3), atol=1e-15)
    assert np.allclose(inst.t2, inst.t2.transpose(1, 0, 3, 2), atol=1e-16)
    assert np.all(np.diff(eo) >= 0) and np.all(np.diff(ev) >= 0)
    assert eo.min() >= -2.0 and eo.max() <= -0.3 and ev.min() >= 0.1 and ev.max() <= 5.0
    assert np.abs(inst.t1).max() < 1e-2 and inst.naux == 3 * (4 + 9)


def test_streams_independent_of_other_sizes():
    a = synth.make_instance(3, 6, seed=4)
    b = synth.make_instance(3, 9, seed=4)
    assert np.array_equal(a.eps_occ, b.eps_occ)


def test_batch_shapes_ranges():
    shapes = synth.batch_shapes(256, 1000)
    assert len(shapes) == 256
    for idx, (o, v, naux, seed) in enumerate(shapes):
        assert 4 <= o <= 16 and 20 <= v <= 120 and naux == 3 * (o + v) and seed == 1000 + idx
    assert len({(o, v) for o, v, _, _ in shapes}) > 100
