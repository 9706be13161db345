"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/tcorr.h declares; host-side validation answers
without touching the device (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_1609_08094_gb300 import _build, tcorr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return tcorr.load()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(tcorr_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"tcorr_create", "tcorr_energy", "tcorr_destroy"} <= names
    for n in names:
        assert hasattr(lib, n), n
    assert set(tcorr.EXPORTS) <= names


def test_status_strings_and_version(lib):
    for i, s in enumerate(tcorr.STATUS):
        assert lib.tcorr_status_string(i).decode() == s
    assert lib.tcorr_status_string(99).decode() == "TCORR_UNKNOWN"
    assert lib.tcorr_version() == 3


def test_invalid_arguments_rejected_before_device_work(lib):
    h = ctypes.c_void_p()
    one = (ctypes.c_double * 1)()
    p = ctypes.cast(one, ctypes.c_void_p)
    # NULL out pointer, zero sizes, NULL arrays: EINVAL without a GPU
    assert lib.tcorr_create(None, 2, 2, p, p, p, p, p, p, p, None, None) == 1
    assert lib.tcorr_create(ctypes.byref(h), 0, 2, p, p, p, p, p, p, p, None, None) == 1
    assert lib.tcorr_create(ctypes.byref(h), 2, 0, p, p, p, p, p, p, p, None, None) == 1
    assert lib.tcorr_create(ctypes.byref(h), 2, 2, p, None, p, p, p, p, p, None, None) == 1
    assert h.value is None
    assert b"NULL" in lib.tcorr_last_error(None) or len(lib.tcorr_last_error(None)) > 0
    bad = tcorr.Opts(prec=7)
    assert lib.tcorr_create(ctypes.byref(h), 2, 2, p, p, p, p, p, p, p, ctypes.byref(bad), None) == 1
    for field, value in (("tune", 2), ("eager", -1), ("wave_mb", -5), ("test_stall", 3),
                         ("host_inputs", 2), ("batch_tasks", -1)):
        o = tcorr.Opts()
        setattr(o, field, value)
        assert lib.tcorr_create(ctypes.byref(h), 2, 2, p, p, p, p, p, p, p, ctypes.byref(o), None) == 1, field
    assert lib.tcorr_destroy(None) == 0
    assert lib.tcorr_num_tasks(None) == -1
    assert lib.tcorr_energy(None, None) == 1


def test_flop_count_definition():
    # 12 v^3 (v+o) per task, i=j=k tasks excluded
    assert tcorr.num_tasks(50) == 22100
    assert tcorr.algorithmic_flops(4, 20) == 12 * 20 ** 3 * 24 * (20 - 4)


def test_batch_arguments_rejected_before_device_work(lib):
    b = ctypes.c_void_p()
    one = (ctypes.c_double * 1)()
    p = ctypes.cast(one, ctypes.c_void_p).value
    good = tcorr.Problem(2, 3, p, p, p, p, p, p, p)
    arr = (tcorr.Problem * 2)(good, tcorr.Problem(2, 3, p, p, p, None, p, p, p))
    assert lib.tcorr_batch_create(None, 1, arr, None, None) == 1
    assert lib.tcorr_batch_create(ctypes.byref(b), 0, arr, None, None) == 1
    assert lib.tcorr_batch_create(ctypes.byref(b), 1, None, None, None) == 1
    assert lib.tcorr_batch_create(ctypes.byref(b), 2, arr, None, None) == 1  # problem 1: NULL t2
    assert b"problem 1" in lib.tcorr_batch_last_error(None)
    zero = (tcorr.Problem * 1)(tcorr.Problem(0, 3, p, p, p, p, p, p, p))
    assert lib.tcorr_batch_create(ctypes.byref(b), 1, zero, None, None) == 1
    big = (tcorr.Problem * 1)(tcorr.Problem(5000, 3, p, p, p, p, p, p, p))
    assert lib.tcorr_batch_create(ctypes.byref(b), 1, big, None, None) == 5
    bad = tcorr.Opts(prec=9)
    assert lib.tcorr_batch_create(ctypes.byref(b), 1, arr, ctypes.byref(bad), None) == 1
    assert b.value is None
    assert lib.tcorr_batch_destroy(None) == 0
    assert lib.tcorr_batch_size(None) == -1
    assert lib.tcorr_batch_device_bytes(None) == -1
    assert lib.tcorr_batch_energy(None, None) == 1
    assert lib.tcorr_batch_plan(None, None, None) == 1
    assert lib.tcorr_batch_tile(None, 0, None) == 1


def test_option_struct_matches_header():
    """The binding's Opts and Problem mirror the C structs field by field."""
    text = open(os.path.join(ROOT, "include", "tcorr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\} tcorr_opts;", text, flags=re.S).group(1)
    fields = re.findall(r"int\s+([a-z_]+)\s*;", body)
    assert fields == [f for f, _ in tcorr.Opts._fields_]
    body = re.search(r"typedef struct \{([^{}]*)\} tcorr_problem;", text, flags=re.S).group(1)
    names = re.findall(r"\*?([a-z_][a-z_0-9]*)[,;]", body)
    assert names == [f for f, _ in tcorr.Problem._fields_]


def test_server_arguments_rejected_before_device_work(lib):
    sv = ctypes.c_void_p()
    assert lib.tcorr_server_create(None, None, 0, None) == 1
    host = tcorr.Opts(host_inputs=1)
    assert lib.tcorr_server_create(ctypes.byref(sv), ctypes.byref(host), 0, None) == 1
    assert lib.tcorr_server_create(ctypes.byref(sv), None, -1, None) == 1
    bad = tcorr.Opts(prec=5)
    assert lib.tcorr_server_create(ctypes.byref(sv), ctypes.byref(bad), 0, None) == 1
    assert sv.value is None
    assert len(lib.tcorr_server_last_error(None)) > 0
    jid = ctypes.c_int64()
    st = ctypes.c_int()
    assert lib.tcorr_server_submit(None, None, ctypes.byref(jid)) == 1
    assert lib.tcorr_server_step(None, None) == 1
    assert lib.tcorr_server_poll(None, 0, ctypes.byref(st), None, None) == 1
    assert lib.tcorr_server_drain(None) == 1
    assert lib.tcorr_server_stats(None, None) == 1
    assert lib.tcorr_server_destroy(None) == 0


def test_mp2_arguments_rejected_before_device_work(lib):
    h = ctypes.c_void_p()
    one = (ctypes.c_double * 1)()
    p = ctypes.cast(one, ctypes.c_void_p)
    # NULL out, sizes < 1, NULL arrays: EINVAL
    assert lib.tcorr_mp2_create(None, 2, 2, 2, p, p, p, None, None) == 1
    assert lib.tcorr_mp2_create(ctypes.byref(h), 0, 2, 2, p, p, p, None, None) == 1
    assert lib.tcorr_mp2_create(ctypes.byref(h), 2, 0, 2, p, p, p, None, None) == 1
    assert lib.tcorr_mp2_create(ctypes.byref(h), 2, 2, 0, p, p, p, None, None) == 1
    assert lib.tcorr_mp2_create(ctypes.byref(h), 2, 2, 2, p, p, None, None, None) == 1
    # an unknown precision is EINVAL; FP64 emulation is not an RI-MP2 precision: EUNSUPPORTED
    bad = tcorr.Opts(prec=7)
    assert lib.tcorr_mp2_create(ctypes.byref(h), 2, 2, 2, p, p, p, ctypes.byref(bad), None) == 1
    oz = tcorr.Opts(prec=tcorr.PREC["fp64_oz"])
    assert lib.tcorr_mp2_create(ctypes.byref(h), 2, 2, 2, p, p, p, ctypes.byref(oz), None) == 5
    assert b"TF32X3" in lib.tcorr_mp2_last_error(None)
    assert h.value is None
    # calls on a NULL handle
    e = (ctypes.c_double * 3)()
    assert lib.tcorr_mp2_energy(None, e) == 1
    assert lib.tcorr_mp2_kernel_times(None, None, None, 0) == 1
    assert lib.tcorr_mp2_device_bytes(None) == -1
    assert lib.tcorr_mp2_destroy(None) == 0


def test_binding_constants_match_the_header():
    """The binding mirrors the header's size limits and routing thresholds."""
    import re
    from paper_1609_08094_gb300 import tcorr
    hdr = open(os.path.join(ROOT, "include", "tcorr.h")).read()
    vals = dict(re.findall(r"#define (TCORR_\w+) ([0-9.e+]+)", hdr))
    assert int(vals["TCORR_NOALLOC_MAX_V"]) == tcorr.NOALLOC_MAX_V
    assert float(vals["TCORR_BF16_MIN_FLOPS"]) == tcorr.BF16_MIN_FLOPS
    assert float(vals["TCORR_MP2_BF16_MIN_TERMS"]) == tcorr.MP2_BF16_MIN_TERMS
