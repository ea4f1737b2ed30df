"""pat_forward_noalloc: the forward model for callers that cannot allocate device memory.

Such callers (an acquisition process with a device memory budget fixed at
start-up, a host program whose device memory belongs to another allocator, a
latency-critical loop that cannot afford the device synchronisation
cudaMalloc may cause) create the plan ahead of time and then run the forward
model with the library's static scratch array instead of a workspace.  The
test calls it through the C ABI twice in a row and compares the traces with
pat_forward's.  It lives in its own file, collected after the other parity
tests (only the slow full-size oracle comparisons follow it), so a failure here
stops a ``-x`` run only after those have run.
"""
import ctypes

import numpy as np
import pytest

import pat_synth as ps
from tests._problems import grid_params, gpu_plan, rel_l2, small_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _noalloc(plan, c, p0, y):
    from paper_2505_08482_gb300 import _binding as B
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return B.lib().pat_forward_noalloc(plan._h, ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(p0.data_ptr()),
                                       ctypes.c_void_p(y.data_ptr()), stream)


def test_noalloc_forward_matches_pat_forward_twice():
    from paper_2505_08482_gb300 import _binding as B
    c, p0, xy = small_case(K=3, nt=150)
    gp = grid_params(40, 150)
    plan = gpu_plan(gp, xy, 3)
    assert plan.workspace_bytes(B.PAT_WS_FORWARD) <= B.PAT_NOALLOC_SCRATCH_BYTES
    cd, pd = _dev(c), _dev(p0)
    ref = plan.forward(cd, pd).cpu().numpy()
    for scale in (1.0, 0.5):     # two calls in a row; the second reuses the scratch
        y = torch.full((3, 150, xy.shape[0]), np.nan, dtype=torch.float32, device="cuda")
        assert _noalloc(plan, cd, _dev(scale * p0), y) == B.PAT_OK
        torch.cuda.synchronize()
        assert rel_l2(y.cpu().numpy(), scale * ref) <= 1e-4


def test_noalloc_forward_headline_grid():
    # 300 x 300 FFT grid (256 x 256 domain): 2 data sets fit in the 16 MiB scratch
    from paper_2505_08482_gb300 import _binding as B
    w = ps.workload("vessels256", 0)
    gp = grid_params(256, 60)
    plan = gpu_plan(gp, w.sensors, 2)
    cd, pd = _dev(w.c_true), _dev(w.p0_true[:2])
    ref = plan.forward(cd, pd).cpu().numpy()
    for _ in range(2):
        y = torch.empty((2, 60, w.m), dtype=torch.float32, device="cuda")
        assert _noalloc(plan, cd, pd, y) == B.PAT_OK
        torch.cuda.synchronize()
        assert rel_l2(y.cpu().numpy(), ref) <= 1e-4


def test_noalloc_rejects_plans_beyond_the_scratch():
    from paper_2505_08482_gb300 import _binding as B
    w = ps.workload("vessels256", 0)
    gp = grid_params(256, 20)
    plan = gpu_plan(gp, w.sensors, 8)
    assert plan.workspace_bytes(B.PAT_WS_FORWARD) > B.PAT_NOALLOC_SCRATCH_BYTES
    y = torch.zeros((8, 20, w.m), dtype=torch.float32, device="cuda")
    rc = _noalloc(plan, _dev(w.c_true), _dev(w.p0_true), y)
    assert rc == B.PAT_EINVAL
    assert b"static scratch" in B.lib().pat_last_error()
    assert float(y.abs().max()) == 0.0
