"""FP64 emulation on the BF16 tensor cores (TCORR_FP64_OZ) against the oracle
at the FP64 tolerance (1e-10 relative), through the C ABI (GPU).  The slice
products are exact, so the error is that of the 5 x 7-bit operand slices
under one scale per operand side; the achieved error is printed."""
import numpy as np
import pytest
import torch

import oracle
from paper_1609_08094_gb300 import synth, tcorr

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1609_08094_gb300 import _build
    _build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("o,v,naux,seed", [
    (4, 20, 72, 1), (3, 16, None, 2), (2, 33, None, 3), (5, 47, None, 4), (3, 130, None, 5),
    (6, 64, None, 6), (2, 270, None, 7), (7, 49, None, 8),
])
def test_oz_matches_oracle(o, v, naux, seed):
    inst = synth.make_instance(o, v, naux, seed)
    ref = oracle.energy(inst)
    with tcorr.Tcorr.from_instance(inst.to("cuda"), prec="fp64_oz") as t:
        e1 = t.energy()
        e2 = t.energy()
    assert e1 == e2
    err = rel(e1[2], ref[2])
    print(f"fp64_oz o={o} v={v}: rel err E(T) {err:.2e}, E4 {rel(e1[0], ref[0]):.2e}, E5 {rel(e1[1], ref[1]):.2e}")
    assert err <= TOL and rel(e1[0], ref[0]) <= TOL
    assert abs(e1[1] - ref[1]) <= TOL * abs(ref[2])


def test_oz_per_task_and_edge_cases():
    inst = synth.make_instance(4, 37, None, 21)
    tasks = oracle.sorted_triples(4)
    ref = oracle.triple_energies(inst, tasks)
    with tcorr.Tcorr.from_instance(inst.to("cuda"), prec="fp64_oz", batch_tasks=3) as t:
        _, per = t.energy_range(0, t.num_tasks, per_task=True)
    scale = np.abs(ref.sum(1)).max()
    assert np.all(np.abs(per.sum(1) - ref.sum(1)) <= TOL * scale)
    one = synth.make_instance(1, 24, None, 3)           # only i = j = k: exact zero
    with tcorr.Tcorr.from_instance(one.to("cuda"), prec="fp64_oz") as t:
        assert t.energy() == (0.0, 0.0, 0.0)
    z = synth.make_instance(3, 20, None, 4)
    z.t1 = np.zeros_like(z.t1)                            # no singles: E5 exactly zero
    with tcorr.Tcorr.from_instance(z.to("cuda"), prec="fp64_oz") as t:
        e4, e5, e = t.energy()
    assert e5 == 0.0 and e == e4


def test_oz_host_inputs_batch_and_server_agree():
    insts = [synth.make_instance(o, v, None, s) for o, v, s in ((3, 40, 31), (5, 29, 32), (2, 75, 33))]
    dev = [i.to("cuda") for i in insts]
    single = []
    for i, d in zip(insts, dev):
        with tcorr.Tcorr.from_instance(d, prec="fp64_oz") as t:
            single.append(t.energy())
        with tcorr.Tcorr.from_instance(i, prec="fp64_oz") as t:      # numpy: copied in
            assert t.energy() == single[-1]
    with tcorr.Batch(dev, prec="fp64_oz") as b:
        e = b.energy()
    for n in range(len(dev)):
        assert tuple(e[n]) == single[n]
    with tcorr.Server(prec="fp64_oz") as s:
        ids = [s.submit(d) for d in dev]
        s.drain()
        for n, jid in enumerate(ids):
            assert s.poll(jid)[1] == single[n]
