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


def test_noalloc_between_checkpointed_forward_and_vjp():
    # a checkpointed pat_forward keeps the last segment's pressure history in its workspace;
    # an allocation-free call in between must make the following pat_vjp recompute it
    # instead of trusting it, so the gradient equals the one without the call in between
    from paper_2505_08482_gb300 import _binding as B
    c, p0, xy = small_case(K=2, nt=120)
    gp = grid_params(40, 120)
    plan = gpu_plan(gp, xy, 2, ckpt_every=16)
    cd, pd = _dev(c), _dev(p0)
    ybar = _dev(ps.rng_for(9).standard_normal((2, 120, xy.shape[0])))
    plan.forward(cd, pd, keep_checkpoints=True)
    g_ref, c_ref = [t.clone() for t in plan.vjp(cd, pd, ybar)]
    plan.forward(cd, pd, keep_checkpoints=True)
    y = torch.empty((2, 120, xy.shape[0]), dtype=torch.float32, device="cuda")
    assert _noalloc(plan, cd, _dev(0.3 * p0), y) == B.PAT_OK
    g, gc = plan.vjp(cd, pd, ybar)
    torch.cuda.synchronize()
    assert rel_l2(g.cpu().numpy(), g_ref.cpu().numpy()) <= 1e-6
    assert rel_l2(gc.cpu().numpy(), c_ref.cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("variant", [0, 3])
def test_noalloc_status_after_a_call(variant):
    # variant 3 stages its rows by bulk copies behind a bounded wait; the status entry point
    # reads that wait's flag from the static array (0: every wait completed)
    from paper_2505_08482_gb300 import _binding as B
    w = ps.workload("plain64", 0)
    gp = grid_params(64, 80)
    plan = gpu_plan(gp, w.sensors, 1)
    plan.variant = variant
    cd, pd = _dev(w.c_true), _dev(w.p0_true)
    ref = plan.forward(cd, pd).cpu().numpy()
    y = torch.empty((1, 80, w.m), dtype=torch.float32, device="cuda")
    assert _noalloc(plan, cd, pd, y) == B.PAT_OK
    flag = ctypes.c_int(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert B.lib().pat_forward_noalloc_status(plan._h, ctypes.byref(flag), stream) == B.PAT_OK
    assert flag.value == 0
    assert rel_l2(y.cpu().numpy(), ref) <= 1e-4


_RESET_CHILD = r'''
import ctypes, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2505_08482_gb300 import _binding as B
from tests._problems import grid_params, small_case

L = ctypes.CDLL(B.LIB)
for name, (res, args) in B.SIGNATURES.items():
    getattr(L, name).restype = res
    getattr(L, name).argtypes = args
rt = ctypes.CDLL("libcudart.so.13")
V = ctypes.c_void_p


def ok(e, what):
    if e != 0:
        raise SystemExit(f"{what} failed: {e} {L.pat_last_error()}")


c, p0, xy = small_case(K=2, nt=100)
gp = grid_params(40, 100)
g = B.PatGrid(gp["n"], gp["pml"], gp["dx"], gp["dt"], gp["nt"], gp["c_ref"], gp["rho0"], gp["pml_alpha"],
              gp["c_bg"])
xy = np.ascontiguousarray(xy, dtype=np.float64)


def to_dev(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    d = V()
    ok(rt.cudaMalloc(ctypes.byref(d), ctypes.c_size_t(a.nbytes)), "cudaMalloc")
    ok(rt.cudaMemcpy(d, a.ctypes.data_as(V), ctypes.c_size_t(a.nbytes), 1), "cudaMemcpy H2D")
    return d


def run():
    plan = V()
    ok(L.pat_plan_create(ctypes.byref(plan), ctypes.byref(g), xy.shape[0],
                         xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 2, 32), "pat_plan_create")
    dc, dp = to_dev(c), to_dev(p0)
    shape = (2, 100, xy.shape[0])
    out = []
    for call in ("noalloc", "forward"):
        y = np.zeros(shape, dtype=np.float32)
        dy = to_dev(y)
        if call == "noalloc":
            ok(L.pat_forward_noalloc(plan, dc, dp, dy, None), "pat_forward_noalloc")
        else:
            nb = L.pat_workspace_bytes(plan, B.PAT_WS_FORWARD)
            ws = V()
            ok(rt.cudaMalloc(ctypes.byref(ws), ctypes.c_size_t(nb)), "cudaMalloc ws")
            ok(L.pat_forward(plan, dc, dp, dy, ws, nb, None), "pat_forward")
        ok(rt.cudaDeviceSynchronize(), "sync")
        ok(rt.cudaMemcpy(y.ctypes.data_as(V), dy, ctypes.c_size_t(y.nbytes), 2), "cudaMemcpy D2H")
        out.append(y)
    L.pat_plan_destroy(plan)
    return out


ok(rt.cudaSetDevice(0), "cudaSetDevice")
a1, b1 = run()
ok(rt.cudaDeviceReset(), "cudaDeviceReset")
ok(rt.cudaSetDevice(0), "cudaSetDevice")
a2, b2 = run()
rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
assert rel(a1, b1) <= 1e-6 and rel(a2, b2) <= 1e-6 and rel(a2, a1) <= 1e-6, (rel(a1, b1), rel(a2, b2), rel(a2, a1))
print("noalloc across device reset ok", rel(a1, b1), rel(a2, b2))
'''


def test_noalloc_after_device_reset(repo_root):
    # a context that is destroyed (cudaDeviceReset) and created again loads the library's device
    # code anew; the allocation-free call must find the static array in the new context.  Runs in a
    # child process that uses the CUDA runtime alone (no PyTorch state to invalidate).
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "-c", _RESET_CHILD, repo_root], capture_output=True, text=True,
                       timeout=300, cwd=repo_root)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "noalloc across device reset ok" in r.stdout
