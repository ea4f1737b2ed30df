"""Host-side argument validation of the C ABI: bad arguments return PAT_EINVAL
with a message before any device work, so these calls need no GPU."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def L():
    from paper_2505_08482_gb300 import build
    from paper_2505_08482_gb300 import _binding as B
    build()
    return B.lib()


@pytest.fixture(scope="module")
def B():
    from paper_2505_08482_gb300 import _binding as B
    return B


def _cfg(B, **kw):
    levels = (ctypes.c_int * 2)(32, 64)
    xy = (ctypes.c_double * 4)(1e-3, 1e-3, 2e-3, 2e-3)
    c = B.PatReconCfg(nlevels=2, levels=levels, L=6.4e-3, dt_data=1.7e-8, nt_data=100, m=2, h_sensor_xy=xy, K=1,
                      cfl=0.3, c_lo=1350.0, c_hi=1750.0, p0_lo=0.0, c_bg=1500.0, rho0=1000.0, pml_alpha=2.0,
                      min_pml=20, mem=20, iters=5, max_halvings=20, ckpt_every=32, rtol=1e-4, alpha0=0.1, c1=1e-4,
                      sigma_p0=0.25, autotune=0, prior_tau=0.0, prior_eta_c=0.0, prior_sigma_c=0.0,
                      prior_eta_p0=0.0, prior_sigma_p0=0.0, persistent=0)
    c._keep = (levels, xy)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


FAKE = ctypes.c_void_p(0x1000)   # never dereferenced: every call below fails validation first


def test_null_plans_and_buffers(L, B):
    for call in (lambda: L.pat_forward(None, FAKE, FAKE, FAKE, FAKE, 1 << 20, None),
                 lambda: L.pat_forward_noalloc(None, FAKE, FAKE, FAKE, None),
                 lambda: L.pat_adjoint_grad(None, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, None, None, FAKE, 1 << 20, None),
                 lambda: L.pat_vjp(None, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, 1 << 20, None),
                 lambda: L.pat_plan_autotune(None, None, 0, None, None),
                 lambda: L.pat_plan_set_graphs(None, 1),
                 lambda: L.pat_plan_set_cluster(None, 1),
                 lambda: L.pat_plan_cluster_capacity(None),
                 lambda: L.pat_status(None, FAKE, ctypes.byref(ctypes.c_int()), None)):
        assert call() == B.PAT_EINVAL
        assert L.pat_last_error()
    assert L.pat_plan_cluster(None) == -1


def test_noalloc_null_arguments(L, B):
    # each buffer NULL in turn (the plan pointer is never dereferenced: the checks come first)
    for args in ((FAKE, None, FAKE, FAKE), (FAKE, FAKE, None, FAKE), (FAKE, FAKE, FAKE, None)):
        assert L.pat_forward_noalloc(*args, None) == B.PAT_EINVAL
        assert b"null argument" in L.pat_last_error()
    flag = ctypes.c_int()
    assert L.pat_forward_noalloc_status(None, ctypes.byref(flag), None) == B.PAT_EINVAL
    assert L.pat_forward_noalloc_status(FAKE, None, None) == B.PAT_EINVAL


def test_multigrid_transfer_arguments(L, B):
    assert L.pat_prolong(None, FAKE, 1, 8, 16, None) == B.PAT_EINVAL
    assert L.pat_prolong(FAKE, None, 1, 8, 16, None) == B.PAT_EINVAL
    for nb, ns, nd in ((0, 8, 16), (1, 0, 16), (1, 8, 0)):
        assert L.pat_prolong(FAKE, FAKE, nb, ns, nd, None) == B.PAT_EINVAL
    assert L.pat_time_interp(None, FAKE, 1, 10, 20, 4, 1e-8, 5e-9, None) == B.PAT_EINVAL
    for K, nts, ntd, m, dts, dtd in ((0, 10, 20, 4, 1e-8, 5e-9), (1, 10, 20, 0, 1e-8, 5e-9),
                                     (1, 10, 20, 4, 0.0, 5e-9), (1, 10, 20, 4, 1e-8, float("nan"))):
        assert L.pat_time_interp(FAKE, FAKE, K, nts, ntd, m, dts, dtd, None) == B.PAT_EINVAL
    assert b"pat_time_interp" in L.pat_last_error()


def test_selftest_and_prior_arguments(L, B):
    assert L.pat_plan_set_persistent(None, 1) == B.PAT_EINVAL
    assert L.pat_plan_persistent(None) == -1
    assert L.pat_selftest_queue(None, FAKE, 1000, None) == B.PAT_EINVAL
    assert L.pat_selftest_queue(FAKE, None, 1000, None) == B.PAT_EINVAL
    assert L.pat_selftest_queue(FAKE, FAKE, 0, None) == B.PAT_EINVAL
    assert L.pat_selftest_wait(None, 1000, None) == B.PAT_EINVAL
    assert L.pat_selftest_wait(FAKE, 0, None) == B.PAT_EINVAL
    assert L.pat_selftest_wait(FAKE, 2000000, None) == B.PAT_EINVAL
    assert L.pat_selftest_bounds(None, None) == B.PAT_EINVAL
    assert L.pat_debug_bounds() == 0   # the release library: checks compiled out
    out = ctypes.c_void_p()
    assert L.pat_prior_create(64, 1e-4, 1.5e-3, 4, None) == B.PAT_EINVAL
    for n, dx, tau, nf in ((1, 1e-4, 1e-3, 1), (600, 1e-4, 1e-3, 1), (64, 0.0, 1e-3, 1), (64, 1e-4, -1.0, 1),
                           (64, 1e-4, 1e-3, 0), (64, 1e-4, float("nan"), 1)):
        assert L.pat_prior_create(n, dx, tau, nf, ctypes.byref(out)) == B.PAT_EINVAL, (n, dx, tau, nf)
        assert not out.value
    assert b"pat_prior_create" in L.pat_last_error()


def test_unet_arguments(L, B):
    out = ctypes.c_void_p()
    for args in ((0, 32, 4, 128, 128, 8), (7, 32, 4, 128, 128, 8), (4, 12, 4, 128, 128, 8),
                 (4, 32, 0, 128, 128, 8), (4, 32, 4, 100, 128, 8), (4, 32, 4, 128, 128, 0)):
        assert L.pat_unet_create(ctypes.byref(out), *args) == B.PAT_EINVAL, args
        assert not out.value


def test_reconstruct_configurations(L, B):
    inst = B.PatInstance(d_y_meas=FAKE, d_w=FAKE, d_c_io=FAKE, d_p0_io=FAKE, K=1)
    assert L.pat_reconstruct_batched(None, 1, ctypes.byref(inst), None) == B.PAT_EINVAL
    assert L.pat_reconstruct_batched(ctypes.byref(_cfg(B)), 0, ctypes.byref(inst), None) == B.PAT_EINVAL
    bad = [dict(nlevels=0), dict(c_hi=1300.0), dict(cfl=0.0), dict(mem=-1), dict(ckpt_every=0), dict(sigma_p0=0.0),
           dict(alpha0=-1.0), dict(prior_tau=-1.0), dict(prior_tau=1e-3), dict(dt_data=0.0), dict(m=0)]
    for kw in bad:
        assert L.pat_reconstruct_batched(ctypes.byref(_cfg(B, **kw)), 1, ctypes.byref(inst), None) == B.PAT_EINVAL, kw
        assert b"pat_reconstruct" in L.pat_last_error()
    levels = (ctypes.c_int * 2)(32, 1)
    assert L.pat_reconstruct_batched(ctypes.byref(_cfg(B, levels=levels)), 1, ctypes.byref(inst), None) == \
        B.PAT_EINVAL
    null_inst = B.PatInstance(d_y_meas=None, d_w=FAKE, d_c_io=FAKE, d_p0_io=FAKE, K=1)
    assert L.pat_reconstruct_batched(ctypes.byref(_cfg(B)), 1, ctypes.byref(null_inst), None) == B.PAT_EINVAL
    assert L.pat_reconstruct(None, FAKE, FAKE, FAKE, FAKE, None, None) == B.PAT_EINVAL
    assert L.pat_reconstruct(ctypes.byref(_cfg(B, K=0)), FAKE, FAKE, FAKE, FAKE, None, None) == B.PAT_EINVAL


def test_sensors_outside_the_grid_or_not_finite(L, B):
    g = B.PatGrid(64, 22, 1e-4, 1e-8, 10, 1750.0, 1000.0, 2.0, 1500.0)
    h = ctypes.c_void_p()
    for x, y in ((-3.0e-3, 3e-3), (3e-3, 9.0e-3), (float("nan"), 3e-3), (3e-3, float("inf"))):
        xy = (ctypes.c_double * 4)(3.2e-3, 3.2e-3, x, y)
        assert L.pat_plan_create(ctypes.byref(h), ctypes.byref(g), 2, xy, 1, 32) == B.PAT_EINVAL, (x, y)
        assert b"sensor 1" in L.pat_last_error() and not h.value
    Ks = (ctypes.c_int * 2)(2, 0)
    xy = (ctypes.c_double * 2)(3.2e-3, 3.2e-3)
    assert L.pat_plan_create_batched(ctypes.byref(h), ctypes.byref(g), 1, xy, 2, Ks, 32) == B.PAT_EINVAL
    assert b"instance 1" in L.pat_last_error()


def _no_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: device allocations succeed")


def test_failed_device_allocations_return_a_status_and_no_object(L, B):
    """Without a device every allocation fails: each creator reports it and hands back nothing."""
    _no_gpu()
    g = B.PatGrid(64, 22, 1e-4, 1e-8, 10, 1750.0, 1000.0, 2.0, 1500.0)
    xy = (ctypes.c_double * 2)(3.2e-3, 3.2e-3)
    h = ctypes.c_void_p()
    rc = L.pat_plan_create(ctypes.byref(h), ctypes.byref(g), 1, xy, 1, 32)
    assert rc in (B.PAT_ENOMEM, B.PAT_ECUDA) and not h.value
    assert b"CUDA error" in L.pat_last_error()
    pr = ctypes.c_void_p()
    rc = L.pat_prior_create(32, 1e-4, 1.5e-3, 2, ctypes.byref(pr))
    assert rc in (B.PAT_ENOMEM, B.PAT_ECUDA) and not pr.value
    net = ctypes.c_void_p()
    rc = L.pat_unet_create(ctypes.byref(net), 2, 8, 1, 16, 16, 1)
    assert rc in (B.PAT_ENOMEM, B.PAT_ECUDA) and not net.value
    assert L.pat_last_error()
