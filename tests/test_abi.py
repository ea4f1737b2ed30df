"""The C ABI: header declarations, exported symbols, host-side validation (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pat.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pat_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2505_08482_gb300 import build
    return build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(pat_[a-z_0-9]+)\b", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_binding_declares_every_header_function():
    from paper_2505_08482_gb300 import _binding as B
    assert sorted(B.exported_symbols()) == declared_functions()


def test_library_loads_and_host_helpers(libpath):
    from paper_2505_08482_gb300 import _binding as B
    L = B.lib()
    assert L.pat_pml_auto(64, 20) == 22
    assert L.pat_pml_auto(256, 20) == 22
    assert L.pat_pml_auto(160, 20) == 20
    assert L.pat_pml_auto(50, 20) == 20        # Ng = 90 = 2 * 3^2 * 5
    from oracle.grid import pml_auto
    for n in range(2, 300, 2):
        assert L.pat_pml_auto(n, 20) == pml_auto(n, 20)
    assert L.pat_pml_auto(63, 20) == -1
    assert L.pat_plan_ng(None) == -1
    assert L.pat_workspace_bytes(None, 0) == 0


def test_plan_create_rejects_bad_grids_before_touching_the_device(libpath):
    from paper_2505_08482_gb300 import _binding as B
    L = B.lib()
    xy = (ctypes.c_double * 2)(0.0032, 0.0032)
    h = ctypes.c_void_p()
    # 64 + 2*21 = 106 = 2 * 53 is not 5-smooth
    g = B.PatGrid(64, 21, 1e-4, 1e-8, 10, 1750.0, 1000.0, 2.0, 1500.0)
    assert L.pat_plan_create(ctypes.byref(h), ctypes.byref(g), 1, xy, 1, 32) == B.PAT_EINVAL
    assert b"5-smooth" in L.pat_last_error()
    # odd grid side: 63 + 2*21 = 105
    g = B.PatGrid(63, 21, 1e-4, 1e-8, 10, 1750.0, 1000.0, 2.0, 1500.0)
    assert L.pat_plan_create(ctypes.byref(h), ctypes.byref(g), 1, xy, 1, 32) == B.PAT_EINVAL
    # 7-smooth but not 5-smooth: 64 + 2*6 = 76 = 4 * 19
    g = B.PatGrid(64, 6, 1e-4, 1e-8, 10, 1750.0, 1000.0, 2.0, 1500.0)
    assert L.pat_plan_create(ctypes.byref(h), ctypes.byref(g), 1, xy, 1, 32) == B.PAT_EINVAL
    g = B.PatGrid(64, 22, -1e-4, 1e-8, 10, 1750.0, 1000.0, 2.0, 1500.0)
    assert L.pat_plan_create(ctypes.byref(h), ctypes.byref(g), 1, xy, 1, 32) == B.PAT_EINVAL
    g = B.PatGrid(64, 22, 1e-4, 1e-8, 0, 1750.0, 1000.0, 2.0, 1500.0)
    assert L.pat_plan_create(ctypes.byref(h), ctypes.byref(g), 1, xy, 1, 32) == B.PAT_EINVAL
    assert L.pat_plan_create(None, ctypes.byref(g), 1, xy, 1, 32) == B.PAT_EINVAL
    assert not h.value
