"""Tensor-core (tcgen05) mixed-precision path against the CPU oracle, through
the C ABI (GPU).  Tolerance: 1e-6 relative on E(T) (Sec. 4 accepts 1e-6 a.u.
for mixed precision); the achieved error is printed."""
import numpy as np
import pytest
import torch

import oracle
from paper_1609_08094_gb300 import synth, tcorr

pytestmark = pytest.mark.gpu
MIXED_TOL = 1e-6


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1609_08094_gb300 import _build
    _build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def energy(inst, prec, **kw):
    dev = inst.to("cuda")
    with tcorr.Tcorr.from_instance(dev, prec=prec, **kw) as t:
        return t.energy()


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("o,v,naux,seed", [
    (4, 20, 72, 1),      # small configuration (o=4, v=20, naux=72)
    (3, 16, None, 2), (2, 33, None, 3), (5, 47, None, 4), (3, 130, None, 5),
    (6, 64, None, 6), (2, 270, None, 7),
])
def test_mixed_matches_oracle(prec, o, v, naux, seed):
    inst = synth.make_instance(o, v, naux, seed)
    ref = oracle.energy(inst)
    got = energy(inst, prec)
    err = rel(got[2], ref[2])
    print(f"{prec} o={o} v={v}: rel err E(T) {err:.2e}, E4 {rel(got[0], ref[0]):.2e}")
    assert err <= MIXED_TOL, (prec, got, ref)
    assert rel(got[0], ref[0]) <= MIXED_TOL


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_mixed_per_task(prec):
    inst = synth.make_instance(4, 37, None, 21)
    tasks = oracle.sorted_triples(4)
    ref = oracle.triple_energies(inst, tasks)
    with tcorr.Tcorr.from_instance(inst.to("cuda"), prec=prec, batch_tasks=3) as t:
        _, per = t.energy_range(0, t.num_tasks, per_task=True)
        e1 = t.energy()
        e2 = t.energy()
    assert e1 == e2  # deterministic (no atomics)
    tot = per.sum(1)
    rt = ref.sum(1)
    scale = np.abs(rt).max()
    assert np.all(np.abs(tot - rt) <= 1e-6 * scale)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_mixed_edge_cases(prec):
    # single occupied: every task is i=j=k, exact zero
    inst = synth.make_instance(1, 24, None, 3)
    assert energy(inst, prec) == (0.0, 0.0, 0.0)
    # zero singles: E5 exactly zero
    inst = synth.make_instance(3, 20, None, 4)
    inst.t1 = np.zeros_like(inst.t1)
    e4, e5, e = energy(inst, prec)
    assert e5 == 0.0 and e == e4


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("o,v,seed", [(4, 20, 1), (3, 16, 2), (3, 130, 5), (2, 270, 7), (6, 160, 8)])
def test_sm_pair_tiles_against_single_sm_tiles_and_oracle(prec, o, v, seed):
    """The SM-pair kernel (2-CTA clusters, M = 256; the default) and the
    single-SM kernel (M = 128) evaluate the same K blocks in the same order
    per output row: both within 1e-6 of the oracle, per task as well.  Shapes:
    v below one 32-row pair of B halves, an odd number of pair tiles (the last
    pair half empty), two N passes (v = 270), and a BF16-operand problem."""
    inst = synth.make_instance(o, v, None, seed)
    tasks = oracle.sorted_triples(o)
    ref = oracle.triple_energies(inst, tasks)
    dev = inst.to("cuda")
    with tcorr.Tcorr.from_instance(dev, prec=prec) as t:
        e_pair, per_pair = t.energy_range(0, t.num_tasks, per_task=True)
    with tcorr.Tcorr.from_instance(dev, prec=prec, single_sm=True) as t:
        e_one, per_one = t.energy_range(0, t.num_tasks, per_task=True)
    tot = ref.sum()
    for e in (e_pair, e_one):
        assert rel(e[2], tot) <= MIXED_TOL, (prec, o, v, e_pair, e_one, tot)
    scale = np.abs(ref.sum(1)).max()
    assert np.all(np.abs(per_pair.sum(1) - ref.sum(1)) <= MIXED_TOL * scale)
    print(f"{prec} o={o} v={v}: pair {rel(e_pair[2], tot):.2e}, single {rel(e_one[2], tot):.2e}, "
          f"identical {e_pair == e_one}")


@pytest.mark.parametrize("single_sm", [False, True])
def test_bounded_wait_expiry_reports_timeout_and_context_survives(single_sm):
    """Failure detection without a fault: the test-only option makes the
    tensor-core producer of CTA 0 withhold one chunk's loads, so the MMA
    issuer's bounded wait expires.  The call must return TCORR_ETIMEOUT (no
    hang, no fault) and the next normal call on the same context must work."""
    import time
    inst = synth.make_instance(3, 40, None, 41)
    dev = inst.to("cuda")
    with tcorr.Tcorr.from_instance(dev, prec="tf32x3", test_stall=True, single_sm=single_sm) as t:
        t0 = time.time()
        with pytest.raises(tcorr.TcorrError) as exc:
            t.energy()
        assert exc.value.status == 4  # TCORR_ETIMEOUT
        assert time.time() - t0 < 60
    ref = oracle.energy(inst)
    got = energy(inst, "tf32x3")
    assert rel(got[2], ref[2]) <= MIXED_TOL
