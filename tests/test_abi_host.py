"""Host-side checks of the C ABI (no GPU needed).

The library must build, load and export every entry point that
include/ppf.h declares; argument validation must return status codes
(never crash) before any device work is attempted.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1511_03599_gb300 import ppf, _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def L():
    if not os.path.exists(ppf.LIB_PATH):
        _build.build()
    return ppf.lib()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ppf_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("ppf_plan", "ppf_execute", "ppf_destroy", "ppf_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, f"not exported: {missing}"


def test_status_strings(L):
    for code, name in ppf.STATUS_NAMES.items():
        assert L.ppf_status_string(code).decode() == name
    assert L.ppf_status_string(99).decode() == "PPF_ERR_UNKNOWN"


def _plan(L, C, T, taps, i=0, o=0, out=True):
    h = ctypes.c_void_p()
    ptr = taps.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if taps is not None else None
    st = L.ppf_plan(ctypes.byref(h) if out else None, C, T, ptr, i, o)
    return st, h


@pytest.mark.parametrize("C,T,i,o,want", [
    (0, 8, 0, 0, 1), (512, 0, 0, 0, 1), (-4, 8, 0, 0, 1),
    (48, 8, 0, 0, 2), (8192, 8, 0, 0, 2), (16, 8, 0, 0, 2), (512, 65, 0, 0, 2), (96, 8, 0, 0, 2),
    (6144, 8, 0, 0, 2), (640, 8, 0, 0, 2),
    (512, 8, 3, 0, 2), (512, 8, 0, 2, 2), (512, 8, -1, 0, 2),
])
def test_plan_rejects_bad_arguments(L, C, T, i, o, want):
    taps = np.ones(max(1, C * T) if C > 0 and T > 0 else 1, dtype=np.float32)
    st, h = _plan(L, C, T, taps, i, o)
    assert st == want, ppf.STATUS_NAMES.get(st)
    assert h.value is None
    assert L.ppf_last_error_message().decode()


def test_plan_rejects_null_pointers(L):
    taps = np.ones(512 * 8, dtype=np.float32)
    assert _plan(L, 512, 8, None)[0] == 1
    assert _plan(L, 512, 8, taps, out=False)[0] == 1


def test_execute_and_destroy_reject_bad_handles(L):
    bogus = ctypes.c_void_p(0x1234560)
    assert L.ppf_execute(None, None, None, 1, None) == 1
    assert L.ppf_execute(bogus, ctypes.c_void_p(16), ctypes.c_void_p(32), 1, None) == 1
    assert L.ppf_execute_host(bogus, ctypes.c_void_p(16), ctypes.c_void_p(32), 1, None) == 1
    assert L.ppf_destroy(None) == 0
    assert L.ppf_destroy(bogus) == 1
    info = (ctypes.c_int * 8)()
    assert L.ppf_plan_info(bogus, info) == 1
    assert L.ppf_check_device(bogus, None) == 1
    assert L.ppf_set_debug_flags(bogus, 1) == 1
    assert L.ppf_probe_rates(None, 5) == 1


def test_python_plan_raises_without_device_or_on_bad_args():
    with pytest.raises((ppf.PPFError, ValueError)):
        ppf.Plan(48, 8, np.ones(48 * 8, np.float32))
    with pytest.raises(ValueError):
        ppf.Plan(512, 8, np.ones(10, np.float32))
    with pytest.raises(ValueError):
        ppf.Plan(512, 8, np.ones(512 * 8, np.float32), in_dtype="u8")
