"""Batched evaluation of many problems of uneven (o, v) (tcorr_batch_*),
through the C ABI (GPU).

Each problem's energies must be bit-identical to a single handle's on the
same problem and precision (the work units of a problem do the same
arithmetic whatever else shares the wave), identical between graph replay and
direct launches and across wave cuts, and within the tolerances against the
oracle: 1e-10 relative for FP64, 1e-6 for the split-precision paths."""
import numpy as np
import pytest
import torch

import oracle
from paper_1609_08094_gb300 import synth, tcorr

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "tf32x3": 1e-6, "bf16x3": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1609_08094_gb300 import _build
    _build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.fixture(scope="module")
def problems():
    # uneven shapes spanning several tiles and ragged tails, plus degenerate ones:
    # o = 1 (only i = j = k tasks, E = 0) and v below one tile edge
    # and one problem above TCORR_BF16_MIN_FLOPS, so that a BF16X3 batch mixes
    # BF16-operand and TF32-operand problems in the same waves
    shapes = [(3, 20, 1), (5, 47, 2), (1, 24, 3), (4, 9, 4), (2, 130, 5), (6, 33, 6),
              (4, 64, 7), (3, 16, 8), (6, 160, 9)]
    insts = [synth.make_instance(o, v, None, seed) for o, v, seed in shapes]
    refs = [oracle.energy(i) for i in insts]
    return insts, refs


def single(inst, prec):
    with tcorr.Tcorr.from_instance(inst.to("cuda"), prec=prec) as t:
        return t.energy()


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x3"])
def test_batch_matches_single_handles_and_oracle(problems, prec):
    insts, refs = problems
    dev = [i.to("cuda") for i in insts]
    with tcorr.Batch(dev, prec=prec) as b:
        e1 = b.energy()   # captures the CUDA graph, then replays it
        e2 = b.energy()   # replay
        waves, launches = b.plan()
    assert np.array_equal(e1, e2)
    assert waves >= 1 and launches == 3 * waves + 1
    for n, inst in enumerate(insts):
        s = single(inst, prec)
        assert tuple(e1[n]) == s, (n, inst.o, inst.v, tuple(e1[n]), s)
        if inst.o == 1:
            assert tuple(e1[n]) == (0.0, 0.0, 0.0)
            continue
        err = rel(e1[n, 2], refs[n][2])
        print(f"{prec} o={inst.o} v={inst.v}: rel err {err:.2e}")
        assert err <= TOL[prec]
        assert rel(e1[n, 0], refs[n][0]) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_wave_cut_and_graph_do_not_change_results(problems, prec):
    insts, _ = problems
    dev = [i.to("cuda") for i in insts]
    with tcorr.Batch(dev, prec=prec) as b:
        ref = b.energy()
        plan_big = b.plan()
    # tiny waves: one task per wave (every wave one segment) ...
    with tcorr.Batch(dev, prec=prec, batch_tasks=1, eager=True) as b:
        e = b.energy()
        plan_one = b.plan()
    assert np.array_equal(e, ref)
    assert plan_one[0] > plan_big[0]
    # ... and a 1 MiB wave budget (segments of several problems share a wave), graph replay
    with tcorr.Batch(dev, prec=prec, wave_mb=1) as b:
        e = b.energy()
        e_again = b.energy()
    assert np.array_equal(e, ref) and np.array_equal(e_again, ref)


def test_measured_tile_choice(problems):
    insts, refs = problems
    dev = [i.to("cuda") for i in insts]
    with tcorr.Batch(dev, prec="tf32x3") as b:
        ref = b.energy()
        model = [b.tile(n) for n in range(len(insts))]
    with tcorr.Batch(dev, prec="tf32x3", tune=True) as b:
        e = b.energy()
        tuned = [b.tile(n) for n in range(len(insts))]
    for (pb, kb) in model + tuned:
        assert pb in (4, 8, 16) and kb == 2
    print("model tiles", model, "measured", tuned)
    # the tile shape only regroups rows of the same GEMMs: same accumulation order
    np.testing.assert_array_equal(e, ref)


def test_batch_host_inputs_and_profile(problems):
    insts, _ = problems
    sub = insts[:3]
    with tcorr.Batch(sub, prec="fp64") as b:   # numpy inputs: copied in
        e_host = b.energy()
    with tcorr.Batch([i.to("cuda") for i in sub], prec="fp64", profile=True) as b:
        e_dev = b.energy()
        kt = b.kernel_times()
        waves, _ = b.plan()
    assert np.array_equal(e_host, e_dev)
    assert kt["gemm"][1] == waves and kt["epilogue"][1] == waves
    assert kt["gemm"][0] > 0


def test_batch_config_shapes_sample():
    """A sample of the 256-molecule workload's shape distribution (o in
    [4, 16], v in [20, 120], naux = 3(o + v)): every problem bit-identical to
    its single handle, and against the oracle where the oracle is cheap."""
    shapes = synth.batch_shapes(8, seed=100)
    insts = [synth.make_instance(o, v, naux, s) for o, v, naux, s in shapes]
    dev = [i.to("cuda") for i in insts]
    for prec in ("fp64", "tf32x3", "bf16x3"):
        with tcorr.Batch(dev, prec=prec) as b:
            e = b.energy()
        for n, inst in enumerate(insts):
            assert tuple(e[n]) == single(inst, prec), (prec, inst.o, inst.v)
            ntask = inst.o * (inst.o + 1) * (inst.o + 2) // 6
            if ntask * inst.v ** 3 * (inst.v + inst.o) <= 3e10:
                ref = oracle.energy(inst)
                assert rel(e[n, 2], ref[2]) <= TOL[prec], (prec, inst.o, inst.v)
