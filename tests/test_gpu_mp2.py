"""RI-MP2 (Sec. 2.1) on the GPU against the oracle, through the C ABI.
FP64 path, tolerance 1e-10 relative: tile edges of 48 virtual indices, so
the shapes below span several tiles with ragged tails, plus o = 1, v below
one tile, naux below one K chunk, host inputs and determinism.  Split
precision on the tensor cores (TF32x3, BF16x3), tolerance 1e-6 relative:
tiles of 128 with ragged tails, one pair, ragged naux, host inputs."""
import numpy as np
import pytest
import torch

import oracle
from paper_1609_08094_gb300 import synth, tcorr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1609_08094_gb300 import _build
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("o,v,naux,seed", [
    (3, 20, 5, 1), (5, 47, 30, 2), (1, 13, 7, 3), (4, 97, 61, 4), (7, 130, 200, 5), (2, 49, 3, 6),
    (9, 200, 420, 7),
])
def test_mp2_matches_oracle(o, v, naux, seed):
    inst = synth.make_mp2_instance(o, v, naux, seed)
    ref = oracle.mp2_energy(inst)
    with tcorr.Mp2.from_instance(inst.to("cuda")) as m:
        e1 = m.energy()
        e2 = m.energy()
    assert e1 == e2                     # deterministic
    for k in range(3):
        assert rel(e1[k], ref[k]) <= 1e-10, (k, e1, ref)
    assert e1[2] < 0


def test_mp2_host_inputs_and_profile():
    inst = synth.make_mp2_instance(6, 75, 90, 11)
    with tcorr.Mp2.from_instance(inst, profile=True) as m:     # numpy: copied in
        e_host = m.energy()
        kt = m.kernel_times()
    with tcorr.Mp2.from_instance(inst.to("cuda")) as m:
        e_dev = m.energy()
    assert e_host == e_dev
    assert kt["gemm"][1] == 1 and kt["gemm"][0] > 0


def test_mp2_same_system_as_the_triples_generator():
    """The RI-MP2 inputs are the occupied-virtual factors of the (T)
    generator's system: E_MP2 from the GPU equals the MP1-amplitude form
    built from that instance's ovov and t2 blocks."""
    o, v = 5, 40
    t = synth.make_instance(o, v, None, 12)
    g = np.asarray(t.ovov).transpose(0, 2, 1, 3)
    e_ref = float(np.sum(np.asarray(t.t2) * (2.0 * g - g.transpose(0, 1, 3, 2))))
    with tcorr.Mp2.from_instance(synth.make_mp2_instance(o, v, None, 12).to("cuda")) as m:
        assert rel(m.energy()[2], e_ref) <= 1e-10


def test_mp2_rejects_fp64_emulation():
    inst = synth.make_mp2_instance(2, 10, 4, 1).to("cuda")
    with pytest.raises(tcorr.TcorrError) as ex:
        tcorr.Mp2.from_instance(inst, prec="fp64_oz")
    assert ex.value.status == 5


MIXED_TOL = 1e-6


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("o,v,naux,seed", [
    (3, 20, 5, 1),         # one tile of 128 with 20 valid rows; naux below one K chunk
    (1, 13, 7, 3),         # a single pair (i = j); BF16X3 runs on TF32 operands here
    (2, 65, 12, 5),        # BF16X3 on TF32 operands (1.5e5 terms)
    (4, 130, 61, 4),       # two tiles, the second with 2 valid rows
    (7, 200, 200, 5),      # ragged naux (kp = 224)
    (2, 300, 420, 7),      # three tiles, the last with 44 valid rows
])
def test_mp2_split_precision_matches_oracle(prec, o, v, naux, seed):
    """Tensor-core RI-MP2 (the paper's mixed-precision variant, split precision)
    against the FP64 oracle at 1e-6 relative, deterministic."""
    inst = synth.make_mp2_instance(o, v, naux, seed)
    ref = oracle.mp2_energy(inst)
    with tcorr.Mp2.from_instance(inst.to("cuda"), prec=prec) as m:
        e1 = m.energy()
        e2 = m.energy()
    assert e1 == e2
    err = rel(e1[2], ref[2])
    print(f"rimp2 {prec} o={o} v={v} naux={naux}: rel err E {err:.2e}, E_J {rel(e1[0], ref[0]):.2e}, "
          f"E_K {abs(e1[1] - ref[1]) / abs(ref[2]):.2e}")
    assert err <= MIXED_TOL
    assert rel(e1[0], ref[0]) <= MIXED_TOL
    assert abs(e1[1] - ref[1]) <= MIXED_TOL * abs(ref[2])


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_mp2_split_precision_host_inputs_and_profile(prec):
    inst = synth.make_mp2_instance(5, 140, 90, 11)
    with tcorr.Mp2.from_instance(inst, prec=prec, profile=True) as m:    # numpy: copied in
        e_host = m.energy()
        kt = m.kernel_times()
    with tcorr.Mp2.from_instance(inst.to("cuda"), prec=prec) as m:
        e_dev = m.energy()
    assert e_host == e_dev
    assert kt["gemm"][1] == 1 and kt["gemm"][0] > 0
