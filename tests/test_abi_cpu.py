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
    assert lib.tcorr_version() == 1


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
    res = tcorr.Opts()
    res.reserved[2] = 1
    assert lib.tcorr_create(ctypes.byref(h), 2, 2, p, p, p, p, p, p, p, ctypes.byref(res), None) == 1
    assert lib.tcorr_destroy(None) == 0
    assert lib.tcorr_num_tasks(None) == -1
    assert lib.tcorr_energy(None, None) == 1


def test_flop_count_definition():
    # 12 v^3 (v+o) per task, i=j=k tasks excluded
    assert tcorr.num_tasks(50) == 22100
    assert tcorr.algorithmic_flops(4, 20) == 12 * 20 ** 3 * 24 * (20 - 4)
