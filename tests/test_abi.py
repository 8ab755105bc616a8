"""The C-ABI library loads and exports every entry point include/crgpu.h declares.

CPU-only: no compute call is made (there may be no GPU here).
"""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1407_7220_gb300 as crg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "crgpu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cr_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(crg.library_path):
        from paper_1407_7220_gb300 import _build
        _build.build()
    return crg.library_path


def test_header_declares_the_binding_names():
    assert sorted(crg.exported_symbols) == _declared()


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing
    L = ctypes.CDLL(built)
    for s in _declared():
        assert hasattr(L, s)


def test_status_strings_and_defaults_without_gpu(built):
    L = crg.lib()
    assert L.cr_status_str(0) == b"ok"
    assert L.cr_status_str(-4).startswith(b"bounded")
    o = crg.default_options()
    assert o.gamma == pytest.approx(1e-2) and o.kkt_every >= 1 and o.momentum == 1


def test_invalid_inputs_rejected_before_any_device_work(built):
    import numpy as np
    L = crg.lib()
    h = ctypes.c_void_p()
    X = np.zeros((3, 5))  # N < n + 1
    y = np.zeros(3)
    st = L.cr_create(X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), y.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     3, 5, None, ctypes.byref(h))
    assert st == crg.CR_EINVAL and not h.value
    assert b"N >= n + 1" in L.cr_last_error(None)
    X = np.ones((10, 2))
    X[3, 1] = np.nan
    y = np.zeros(10)
    st = L.cr_create(X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), y.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     10, 2, None, ctypes.byref(h))
    assert st == crg.CR_EINVAL
