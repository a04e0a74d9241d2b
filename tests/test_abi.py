"""The C-ABI library builds, loads and exports every entry point include/*.h
declares; argument errors that are decided on the host come back as the
documented status codes (no GPU needed for any of this)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(qft_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1301_0763_gb300 import build
    path = build.build()
    from paper_1301_0763_gb300 import qft
    return qft.load_library(path)


def test_header_declares_the_documented_entry_points():
    names = _declared_functions()
    for n in ["qft_plan_create", "qft_plan_create_ragged", "qft_execute", "qft_execute_forward",
              "qft_execute_inverse", "qft_execute_backward", "qft_plan_destroy", "qft_status_string"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_argument_errors(lib):
    from paper_1301_0763_gb300 import qft
    h = ctypes.c_void_p()
    assert lib.qft_plan_create(None, 16, 1, 0, 0, 0) == -5            # null out
    assert lib.qft_plan_create(ctypes.byref(h), 12, 1, 0, 0, 0) == -1  # not a power of two
    assert lib.qft_plan_create(ctypes.byref(h), 1, 1, 0, 0, 0) == -1
    assert lib.qft_plan_create(ctypes.byref(h), 1 << 30, 1, 0, 0, 0) == -1
    assert lib.qft_plan_create(ctypes.byref(h), 16, -1, 0, 0, 0) == -2
    assert lib.qft_plan_create(ctypes.byref(h), 16, 1, 7, 0, 0) == -3
    assert lib.qft_plan_create(ctypes.byref(h), 16, 1, 1, 1, 0) == -3  # R2C fp16 unsupported
    assert lib.qft_plan_create(ctypes.byref(h), 16, 1, 0, 0, 8) == -9  # unknown flag bit
    assert lib.qft_execute(None, 0, None, None, None) == -5
    assert lib.qft_plan_destroy(None) == 0
    for code in [0, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10]:
        s = qft.status_string(code)
        assert s and s != "unknown status"
