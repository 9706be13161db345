"""Mixed-precision E(T) across the served workload's size range (GPU).

44 seeded problems: 20 small ones (o = 4..10, v = 20..64, where the BF16
split's residual averages least) and 24 spread over the whole served range
(o = 4..40, v = 20..300).  Each is evaluated in TF32X3 and BF16X3 through
the C ABI and must lie within 1e-6 relative of the FP64 reference (Sec. 4's
mixed-precision tolerance): the CPU oracle itself where it finishes in a few
seconds, else the FP64-emulation GPU path (held to 1e-10 of the oracle by
test_gpu_oz.py).  BF16X3 problems below TCORR_BF16_MIN_FLOPS run on TF32
operands, so their BF16X3 and TF32X3 results must be bit-identical; above it
they must differ (BF16 operands really used).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1609_08094_gb300 import synth, tcorr

pytestmark = pytest.mark.gpu
MIXED_TOL = 1e-6
ORACLE_MAX_FLOPS = 4e11
SHAPES = (synth.batch_shapes(20, 300, o_range=(4, 10), v_range=(20, 64))
          + synth.batch_shapes(24, 100, o_range=(4, 40), v_range=(20, 300)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1609_08094_gb300 import _build
    _build.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def energy(dev, prec):
    with tcorr.Tcorr.from_instance(dev, prec=prec) as t:
        return np.array(t.energy())


@pytest.mark.parametrize("o,v,naux,seed", SHAPES)
def test_mixed_error_across_the_served_range(o, v, naux, seed):
    dev = synth.make_instance(o, v, naux, seed, device="cuda")
    fl = tcorr.algorithmic_flops(o, v)
    if fl <= ORACLE_MAX_FLOPS:
        ref, src = np.array(oracle.energy(dev.numpy())), "oracle"
    else:
        ref, src = energy(dev, "fp64_oz"), "fp64_oz"
    e_tf = energy(dev, "tf32x3")
    e_bf = energy(dev, "bf16x3")
    err_tf = abs(e_tf[2] - ref[2]) / abs(ref[2])
    err_bf = abs(e_bf[2] - ref[2]) / abs(ref[2])
    print(f"o={o} v={v} ({fl:.1e} flop) vs {src}: tf32x3 {err_tf:.2e}, bf16x3 {err_bf:.2e}")
    assert err_tf <= MIXED_TOL
    assert err_bf <= MIXED_TOL
    if fl < tcorr.BF16_MIN_FLOPS:
        assert np.array_equal(e_bf, e_tf)       # routed to TF32 operands
    else:
        assert not np.array_equal(e_bf, e_tf)   # BF16 operands
    del dev
    torch.cuda.empty_cache()


def test_mp2_bf16_routing_threshold():
    """RI-MP2 BF16X3 below TCORR_MP2_BF16_MIN_TERMS uses TF32 operands (results
    identical to TF32X3); above it BF16 operands; both within 1e-6."""
    for o, v, naux, seed in ((1, 13, 7, 3), (2, 65, 12, 5), (7, 200, 200, 5)):
        inst = synth.make_mp2_instance(o, v, naux, seed)
        ref = oracle.mp2_energy(inst)
        e = {}
        for p in ("tf32x3", "bf16x3"):
            with tcorr.Mp2.from_instance(inst.to("cuda"), prec=p) as m:
                e[p] = m.energy()
            assert abs(e[p][2] - ref[2]) <= MIXED_TOL * abs(ref[2]), (o, v, naux, p)
        terms = o * (o + 1) // 2 * v * v * naux
        assert (e["bf16x3"] == e["tf32x3"]) == (terms < tcorr.MP2_BF16_MIN_TERMS), (o, v, naux)
