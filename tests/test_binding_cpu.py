"""The ctypes binding's own argument checks, on the host (no GPU): shapes,
dtypes, contiguity and precision names are rejected in Python before the
library is called; valid host arrays reach tcorr_create, which on a machine
without a GPU answers with a status instead of crashing."""
import numpy as np
import pytest

from paper_1609_08094_gb300 import _build, synth, tcorr


@pytest.fixture(scope="module")
def inst():
    _build.build()
    tcorr.load()
    return synth.make_instance(3, 5, None, 1)


def args_of(inst):
    return [inst.o, inst.v] + [np.ascontiguousarray(a) for a in inst.arrays()]


def test_shape_dtype_and_contiguity_are_checked(inst):
    base = args_of(inst)
    bad_shape = list(base)
    bad_shape[5] = base[5][:, :, :, :-1]                  # t2 missing a column
    with pytest.raises(ValueError, match="t2: expected shape"):
        tcorr.Tcorr(*bad_shape)
    bad_dtype = list(base)
    bad_dtype[6] = base[6].astype(np.float32)             # vvvo in float32
    with pytest.raises(ValueError, match="vvvo: needs a C-contiguous float64"):
        tcorr.Tcorr(*bad_dtype)
    bad_layout = list(base)
    bad_layout[4] = np.asfortranarray(base[4])            # t1 column-major
    with pytest.raises(ValueError, match="t1: needs a C-contiguous float64"):
        tcorr.Tcorr(*bad_layout)


def test_precision_names(inst):
    assert tcorr._prec("BF16X3") == 2 and tcorr._prec("fp64_oz") == 3 and tcorr._prec(1) == 1
    with pytest.raises(ValueError, match="unknown precision"):
        tcorr.Tcorr(*args_of(inst), prec="fp16")
    m = synth.make_mp2_instance(2, 5, 4, 1)
    with pytest.raises(ValueError, match="unknown precision"):
        tcorr.Mp2.from_instance(m, prec="int8")


def test_mp2_shapes_are_checked():
    m = synth.make_mp2_instance(2, 5, 4, 1)
    with pytest.raises(ValueError, match="C: expected shape"):
        tcorr.Mp2(m.o, m.v, m.naux + 1, m.eps_occ, m.eps_vir, m.C)


def test_valid_host_arrays_reach_the_library(inst):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: creation would succeed (covered by the GPU tests)")
    with pytest.raises(tcorr.TcorrError) as ex:
        tcorr.Tcorr(*args_of(inst))
    assert ex.value.status == 3                            # TCORR_ECUDA: no device
