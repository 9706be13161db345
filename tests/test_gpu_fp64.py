"""FP64 CUDA path against the CPU oracle, through the C ABI (GPU)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1609_08094_gb300 import synth, tcorr

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-10


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1609_08094_gb300 import _build
    _build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def run(inst, **kw):
    dev = inst.to("cuda")
    with tcorr.Tcorr.from_instance(dev, **kw) as t:
        return t.energy()


@pytest.mark.parametrize("o,v,naux,seed", [
    (4, 20, 72, 1),        # small configuration (o=4, v=20, naux=72)
    (3, 7, None, 2), (5, 13, None, 3), (2, 33, None, 4), (6, 17, None, 5),
    (7, 9, None, 6), (3, 40, None, 7), (1, 5, None, 8), (4, 1, None, 9), (2, 2, None, 10),
    (3, 130, None, 14),    # a tiles of 32: the last holds 2 of its 32 values (as at v = 450)
])
def test_fp64_matches_oracle(o, v, naux, seed):
    inst = synth.make_instance(o, v, naux, seed)
    ref = oracle.energy(inst)
    got = run(inst)
    if o == 1 or v == 1:
        *_, scale = oracle.bruteforce(inst, with_scale=True)
        assert abs(got[2]) <= 1e-12 * scale + 1e-300
        return
    for g, r in zip(got, ref):
        assert rel(g, r) <= FP64_TOL, (got, ref)


def test_fp64_per_task_and_ranges():
    inst = synth.make_instance(5, 19, None, 11)
    tasks = oracle.sorted_triples(5)
    ref = oracle.triple_energies(inst, tasks)
    dev = inst.to("cuda")
    with tcorr.Tcorr.from_instance(dev, batch_tasks=4) as t:
        assert t.num_tasks == len(tasks)
        for n in (0, 7, len(tasks) - 1):
            assert t.task(n) == tuple(tasks[n])
        full, per = t.energy_range(0, t.num_tasks, per_task=True)
        scale = np.abs(ref).max()
        assert np.all(np.abs(per - ref) <= FP64_TOL * scale)
        # split ranges sum to the full energy
        a = t.energy_range(0, 13)
        b = t.energy_range(13, t.num_tasks - 13)
        assert rel(a[2] + b[2], full[2]) <= 1e-13
        with pytest.raises(tcorr.TcorrError):
            t.energy_range(3, t.num_tasks)


def test_fp64_deterministic_and_batch_invariant():
    inst = synth.make_instance(4, 26, None, 12).to("cuda")
    with tcorr.Tcorr.from_instance(inst, batch_tasks=1) as t:
        e1 = t.energy()
        e2 = t.energy()
    with tcorr.Tcorr.from_instance(inst, batch_tasks=7) as t:
        e3 = t.energy()
    assert e1 == e2  # bitwise
    assert rel(e1[2], e3[2]) <= 1e-14


def test_host_inputs_equal_device_inputs():
    inst = synth.make_instance(4, 21, None, 13)
    with tcorr.Tcorr.from_instance(inst) as t:  # numpy arrays: staged by the library
        eh = t.energy()
    ed = run(inst)
    assert eh == ed


def test_zero_singles_zero_e5_exact():
    inst = synth.make_instance(3, 15, None, 14)
    inst.t1 = np.zeros_like(inst.t1)
    e4, e5, e = run(inst)
    assert e5 == 0.0 and e == e4


def test_out_of_memory_reported():
    # a footprint far above HBM must give ENOMEM, not a crash
    o, v = 60, 2500
    small = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib = tcorr.load()
    import ctypes
    h = ctypes.c_void_p()
    p = ctypes.c_void_p(small.data_ptr())
    st = lib.tcorr_create(ctypes.byref(h), o, v, p, p, p, p, p, p, p, None, None)
    assert st == 2 and h.value is None
