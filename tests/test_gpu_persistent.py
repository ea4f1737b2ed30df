"""Persistent forward sweep (pat_plan_set_persistent) against the launched passes and the oracle.

The persistent sweep runs the initial pass and every time step of all data sets
of a plan in one launch: CTAs take (pass, data set, tile) work items from a
counter and each item waits only for its own data set's earlier passes.  It
computes each element with the same pass bodies and factorisations as kernel
variant 0, compiled into another kernel (the compiler may fuse a different
product of a complex multiply into an FMA there), so traces, checkpoints and
gradients agree with variant 0's to a few FP32 roundings (1e-6 relative) and
with the FP64 oracle within the FP32 tolerance; a batched plan in persistent
form is bit-identical to its instances run one by one in persistent form.
"""
import numpy as np
import pytest

import pat_synth as ps
from tests._problems import grid_params, gpu_plan, oracle_grid, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _case(n, K, seed):
    rng = ps.rng_for(seed)
    c = ps.ellipse_phantom(n, 3, rng)
    p0 = np.stack([ps.blob_p0(n, 4, rng, sigma_cells=(1.5, 3.0)) for _ in range(K)])
    return c, p0


# every grid side with a compiled persistent sweep: Ng = n + 2 P
@pytest.mark.parametrize("n,nt", [(64, 140), (104, 90), (136, 80), (160, 70), (200, 60), (256, 50)])
def test_persistent_forward_is_bit_identical_and_matches_oracle(n, nt):
    from oracle.forward import forward
    from oracle.sensors import sensor_matrix
    from paper_2505_08482_gb300 import _binding as B
    K = 3
    c, p0 = _case(n, K, n)
    xy = ps.rng_for(n + 1).uniform(0.3 * n, 0.7 * n, size=(48, 2)) * 1e-4
    gp = grid_params(n, nt)
    plan = gpu_plan(gp, xy, K)
    assert plan.ng in (108, 144, 180, 200, 240, 300)
    plan.variant = 0
    ref = plan.forward(_dev(c), _dev(p0)).clone()
    plan.persistent = True
    assert plan.persistent
    y = plan.forward(_dev(c), _dev(p0))
    torch.cuda.synchronize()
    # no bounded wait gave up (the forward workspace has no objective, so only these bits count)
    assert plan.status(kind=0) & (B.PAT_STATUS_WAIT | B.PAT_STATUS_QUEUE) == 0
    assert rel_l2(y.cpu().numpy(), ref.cpu().numpy()) <= 1e-6
    g = oracle_grid(gp)
    assert rel_l2(y.cpu().numpy(), forward(g, c, p0, sensor_matrix(g, xy))) <= 1e-4


@pytest.mark.parametrize("ckpt", [7, 32, 1000])
def test_persistent_gradient_equals_launched(ckpt):
    """Checkpoints and the last segment's history written by the persistent sweep feed the
    reverse sweep exactly as the launched sweep's do."""
    n, K, nt = 64, 2, 150
    c, p0 = _case(n, K, 5)
    xy = ps.circle_sensors(n, 32, 1e-4)
    gp = grid_params(n, nt)
    plan = gpu_plan(gp, xy, K, ckpt_every=ckpt)
    plan.variant = 0
    ym = _dev(ps.rng_for(6).standard_normal((K, nt, 32)) * 0.05)
    w = _dev(np.array([1.0, 2.5]))
    c0, p00 = _dev(np.full((n, n), 1495.0)), _dev(0.5 * p0)
    J0, g0, gc0 = [t.clone() for t in plan.adjoint_grad(c0, p00, ym, w)]
    plan.persistent = True
    J1, g1, gc1 = plan.adjoint_grad(c0, p00, ym, w)
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert abs(J1.item() - J0.item()) <= 1e-6 * abs(J0.item())
    assert rel_l2(g1.cpu().numpy(), g0.cpu().numpy()) <= 1e-5
    assert rel_l2(gc1.cpu().numpy(), gc0.cpu().numpy()) <= 1e-5
    # vjp after a persistent forward that kept the checkpoints
    ybar = _dev(ps.rng_for(7).standard_normal((K, nt, 32)))
    plan.persistent = False
    plan.forward(_dev(c), _dev(p0), keep_checkpoints=True)
    v0 = [t.clone() for t in plan.vjp(_dev(c), _dev(p0), ybar)]
    plan.persistent = True
    plan.forward(_dev(c), _dev(p0), keep_checkpoints=True)
    v1 = plan.vjp(_dev(c), _dev(p0), ybar)
    assert rel_l2(v1[0].cpu().numpy(), v0[0].cpu().numpy()) <= 1e-5
    assert rel_l2(v1[1].cpu().numpy(), v0[1].cpu().numpy()) <= 1e-5


def test_persistent_batched_plan_and_graphs():
    """A batched plan (instances with their own c and K) in one persistent launch, also
    replayed from a CUDA graph: bit-identical to each instance alone in persistent form."""
    n = 64
    Ks = [1, 3, 2, 4]
    xy = ps.circle_sensors(n, 24, 1e-4)
    gp = grid_params(n, 100)
    cs, p0s = zip(*[_case(n, K, 30 + i) for i, K in enumerate(Ks)])
    plan = gpu_plan(gp, xy, Ks)
    plan.variant = 0
    cb, pb = _dev(np.stack(cs)), _dev(np.concatenate(p0s))
    launched = plan.forward(cb, pb).clone()
    plan.persistent = True
    ref = plan.forward(cb, pb).clone()
    assert rel_l2(ref.cpu().numpy(), launched.cpu().numpy()) <= 1e-6
    k0 = 0
    for i, K in enumerate(Ks):
        one = gpu_plan(gp, xy, K)
        one.persistent = True
        assert torch.equal(one.forward(_dev(cs[i]), _dev(p0s[i])), ref[k0:k0 + K])
        k0 += K
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    plan.set_graphs(True)
    with torch.cuda.stream(stream):
        ys = [plan.forward(cb, pb, stream=stream).clone() for _ in range(3)]
    torch.cuda.synchronize()
    for y in ys:
        assert torch.equal(y, ref)


def test_persistent_nt1_and_generic_side():
    from paper_2505_08482_gb300 import _binding as B
    n = 64
    c, p0 = _case(n, 2, 8)
    xy = ps.circle_sensors(n, 16, 1e-4)
    plan = gpu_plan(grid_params(n, 1), xy, 2)
    plan.variant = 0
    ref = plan.forward(_dev(c), _dev(p0)).clone()
    plan.persistent = True
    assert rel_l2(plan.forward(_dev(c), _dev(p0)).cpu().numpy(), ref.cpu().numpy()) <= 1e-6
    gen = gpu_plan(grid_params(40, 20), ps.circle_sensors(40, 8, 1e-4), 1)   # Ng 80: no persistent sweep
    with pytest.raises(B.PatError):
        gen.persistent = True
    assert not gen.persistent


def test_queue_wait_gives_up_and_reports():
    """The dependency wait of the persistent sweep, on an item nothing produces, gives up after
    its limit, sets PAT_STATUS_QUEUE and the abort flag; the context stays usable."""
    import ctypes
    from paper_2505_08482_gb300 import _binding as B
    q = torch.full((3,), 7, dtype=torch.int32, device="cuda")
    st = torch.zeros((1,), dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert B.lib().pat_selftest_queue(ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(st.data_ptr()), 20000,
                                      stream) == B.PAT_OK
    torch.cuda.synchronize()
    assert int(st.item()) & B.PAT_STATUS_QUEUE
    assert q.tolist()[1] == 1 and q.tolist()[2] == 0
    x = torch.arange(10, device="cuda").sum()
    assert int(x.item()) == 45
