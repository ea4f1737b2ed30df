"""The C ABI from plain C: include/pat.h compiles as C99 and a C caller links against libpat.so
and the CUDA runtime (no GPU needed; tests/test_gpu_c_caller.py runs it)."""
import shutil

import pytest


def test_c_caller_compiles_and_links(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    import paper_2505_08482_gb300 as pkg
    from tests.c.build_c_caller import build_c_caller
    pkg.build()
    diag = build_c_caller(str(tmp_path / "pat_c_caller"))
    assert diag.strip() == "", diag
    assert (tmp_path / "pat_c_caller").exists()
