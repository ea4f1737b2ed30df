"""The debug build's device-side bounds checks (libpat_debug.so, -DPAT_DEBUG_BOUNDS).

A child process loads the bounds-checked library: its self-test must report a check on an
index one past the end through PAT_STATUS_BOUNDS, no check may fail on correct plans (generic
and fixed-size passes, ragged tiles, ragged checkpoint segments, the TMA-staged variant), and
its traces and gradients must equal those of the release library, whose checks compile to
nothing (the same arithmetic).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_checks_and_matches_release(tmp_path):
    from tests._debug_bounds_cases import run_cases
    from paper_2505_08482_gb300 import _binding as B
    assert B.lib().pat_debug_bounds() == 0
    rel = run_cases()
    assert int(rel["selftest_status"][0]) == 0   # release: the check is compiled out
    out = str(tmp_path / "debug.npz")
    env = dict(os.environ, PAT_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_debug_bounds_cases.py"), out], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    dbg = dict(np.load(out))
    assert int(dbg["debug_bounds"]) == 1
    assert int(dbg["selftest_status"][0]) == B.PAT_STATUS_BOUNDS
    for key, v in rel.items():
        if key.endswith("_status"):
            if key != "selftest_status":
                assert (dbg[key] & B.PAT_STATUS_BOUNDS).sum() == 0 and (v & B.PAT_STATUS_BOUNDS).sum() == 0, key
            continue
        if key == "debug_bounds":
            continue
        a, b = dbg[key].astype(np.float64), v.astype(np.float64)
        assert np.isfinite(a).all()
        err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert err <= 1e-6, (key, err)
