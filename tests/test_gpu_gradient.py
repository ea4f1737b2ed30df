"""GPU gradient (pat_adjoint_grad, pat_vjp) against the FP64 oracle.

Tolerances: J to 1e-4 relative; dJ/dp0 and dJ/dc to 1e-3 relative L2.
"""
import numpy as np
import pytest

from tests._problems import grid_params, oracle_grid, gpu_plan, rel_l2, small_case
import pat_synth as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _oracle(gp, c, p0, xy, ym, w):
    from oracle.adjoint import adjoint_grad
    from oracle.sensors import sensor_matrix
    g = oracle_grid(gp)
    return adjoint_grad(g, c, p0, sensor_matrix(g, xy), ym, w)


def _data(gp, c_true, p0_true, xy, seed):
    from oracle.forward import forward
    from oracle.sensors import sensor_matrix
    g = oracle_grid(gp)
    y = forward(g, c_true, p0_true, sensor_matrix(g, xy))
    y = ps.add_noise(y, ps.rng_for(seed))
    return y, ps.noise_weights(y)


@pytest.mark.parametrize("ckpt", [32, 400])
def test_gradient_plain64_matches_oracle(ckpt):
    w = ps.workload("plain64", 0)
    gp = grid_params(64, 400)
    ym, wt = _data(gp, w.c_true, w.p0_true, w.sensors, 1)
    c0 = np.full((64, 64), 0.5 * (w.c_true.min() + w.c_true.max()))
    p0 = 0.6 * w.p0_true
    J, gp0, gc = _oracle(gp, c0, p0, w.sensors, ym, wt)
    plan = gpu_plan(gp, w.sensors, 1, ckpt_every=ckpt)
    Jg, gp0g, gcg = plan.adjoint_grad(_dev(c0), _dev(p0), _dev(ym), _dev(wt))
    assert abs(Jg.item() - J) <= 1e-4 * J
    assert rel_l2(gp0g.cpu().numpy(), gp0) <= 1e-3
    assert rel_l2(gcg.cpu().numpy(), gc) <= 1e-3


def test_gradient_ragged_multi_k_partial_segments():
    c, p0, xy = small_case(K=3, nt=150)
    gp = grid_params(40, 150)
    ym, wt = _data(gp, c, p0, xy, 2)
    c0 = np.full((40, 40), 1510.0)
    J, gp0, gc = _oracle(gp, c0, 0.5 * p0, xy, ym, wt)
    plan = gpu_plan(gp, xy, 3, ckpt_every=7)     # 22 segments, the last one of 3 steps
    Jg, gp0g, gcg = plan.adjoint_grad(_dev(c0), _dev(0.5 * p0), _dev(ym), _dev(wt))
    assert abs(Jg.item() - J) <= 1e-4 * J
    assert rel_l2(gp0g.cpu().numpy(), gp0) <= 1e-3
    assert rel_l2(gcg.cpu().numpy(), gc) <= 1e-3


def test_checkpointing_matches_full_history():
    c, p0, xy = small_case(K=2, nt=130)
    gp = grid_params(40, 130)
    ym, wt = _data(gp, c, p0, xy, 3)
    c0 = np.full((40, 40), 1490.0)
    res = []
    for s in (5, 32, 130, 1000):
        plan = gpu_plan(gp, xy, 2, ckpt_every=s)
        J, a, b = plan.adjoint_grad(_dev(c0), _dev(0.7 * p0), _dev(ym), _dev(wt))
        res.append((J.item(), a.cpu().numpy(), b.cpu().numpy()))
    for J, a, b in res[1:]:
        assert abs(J - res[0][0]) <= 1e-6 * res[0][0]
        assert rel_l2(a, res[0][1]) <= 1e-5
        assert rel_l2(b, res[0][2]) <= 1e-5


def test_vjp_after_forward_equals_gradient_and_is_repeatable():
    c, p0, xy = small_case(K=2, nt=90)
    gp = grid_params(40, 90)
    ym, wt = _data(gp, c, p0, xy, 4)
    plan = gpu_plan(gp, xy, 2, ckpt_every=16)
    cd, pd = _dev(np.full((40, 40), 1520.0)), _dev(0.4 * p0)
    J, a, b = plan.adjoint_grad(cd, pd, _dev(ym), _dev(wt))
    y = plan.forward(cd, pd, keep_checkpoints=True)
    r = (y - _dev(ym)) * _dev(wt)[:, None, None]
    a2, b2 = plan.vjp(cd, pd, r)
    a3, b3 = plan.vjp(cd, pd, r)     # second call recomputes every segment
    for x, y_ in ((a2, a), (b2, b), (a3, a), (b3, b)):
        assert rel_l2(x.cpu().numpy(), y_.cpu().numpy()) <= 1e-5


def test_dot_product_fp32():
    # <A x, r> = <x, A^T r> for A: p0 -> y at fixed c (vjp without the c part)
    c, p0, xy = small_case(K=2, nt=100)
    gp = grid_params(40, 100)
    plan = gpu_plan(gp, xy, 2, ckpt_every=10)
    rng = ps.rng_for(9)
    x = _dev(rng.standard_normal((2, 40, 40)))
    r = _dev(rng.standard_normal((2, 100, xy.shape[0])))
    cd = _dev(c)
    Ax = plan.forward(cd, x, keep_checkpoints=True)
    ATr, _ = plan.vjp(cd, x, r)
    lhs = float((Ax.double() * r.double()).sum())
    rhs = float((x.double() * ATr.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * float(Ax.double().norm() * r.double().norm())


def test_single_sample_gradient():
    c, p0, xy = small_case(K=2, nt=1)
    gp = grid_params(40, 1)
    ym = ps.rng_for(3).standard_normal((2, 1, xy.shape[0]))
    wt = np.array([2.0, 0.5])
    J, gp0, gc = _oracle(gp, c, p0, xy, ym, wt)
    plan = gpu_plan(gp, xy, 2)
    Jg, a, b = plan.adjoint_grad(_dev(c), _dev(p0), _dev(ym), _dev(wt))
    assert abs(Jg.item() - J) <= 1e-5 * J
    assert rel_l2(a.cpu().numpy(), gp0) <= 1e-6
    assert np.abs(b.cpu().numpy()).max() == 0.0


def test_nonfinite_flag():
    c, p0, xy = small_case(K=1, nt=20)
    gp = grid_params(40, 20)
    plan = gpu_plan(gp, xy, 1)
    ym = np.zeros((1, 20, xy.shape[0]))
    ym[0, 3, 2] = np.nan
    plan.adjoint_grad(_dev(c), _dev(p0[:1]), _dev(ym), _dev(np.ones(1)))
    assert plan.nonfinite()
    plan.adjoint_grad(_dev(c), _dev(p0[:1]), _dev(np.zeros_like(ym)), _dev(np.ones(1)))
    assert not plan.nonfinite()


@pytest.mark.parametrize("variant", [-1, 0, 3])
def test_vjp_with_stale_history_recomputes_last_segment(variant):
    # Nt - 1 = 2 s: the last segment holds the single level Nt - 1, restored from the
    # checkpoint taken when the forward sweep reaches it
    n, nt, s = 64, 33, 16
    xy = ps.circle_sensors(n, 16, 1e-4)
    gp = grid_params(n, nt)
    rng = ps.rng_for(31)
    c = _dev(ps.ellipse_phantom(n, 3, rng))
    p0 = _dev(np.stack([ps.vessel_p0(n, rng) for _ in range(2)]))
    ybar = _dev(rng.standard_normal((2, nt, 16)))
    plan = gpu_plan(gp, xy, 2, ckpt_every=s)
    plan.variant = variant
    plan.forward(c, p0, keep_checkpoints=True)
    g1 = [t.clone() for t in plan.vjp(c, p0, ybar)]          # history of the last segment kept
    plan.forward(c, p0, keep_checkpoints=True)
    plan.forward(c, p0)                                      # forward workspace: history now stale
    g2 = plan.vjp(c, p0, ybar)                               # last segment recomputed
    assert torch.equal(g1[0], g2[0]) and torch.equal(g1[1], g2[1])
    from paper_2505_08482_gb300 import _binding as B
    assert not plan.status() & B.PAT_STATUS_WAIT            # no bounded wait gave up


def test_bounded_wait_gives_up_and_reports():
    # a wait that nothing completes ends after its limit, sets PAT_STATUS_WAIT, and the
    # context stays usable for the solver afterwards
    from paper_2505_08482_gb300 import _binding as B
    st = torch.zeros((), dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    B.check(B.lib().pat_selftest_wait(st.data_ptr(), 2000, s.cuda_stream), "pat_selftest_wait")
    torch.cuda.synchronize()
    assert st.item() & B.PAT_STATUS_WAIT
    with pytest.raises(B.PatError):
        B.check(B.lib().pat_selftest_wait(st.data_ptr(), 0, s.cuda_stream), "pat_selftest_wait")
    c, p0, xy = small_case(K=1, nt=40)
    plan = gpu_plan(grid_params(40, 40), xy, 1)
    y = plan.forward(_dev(c), _dev(p0))
    assert torch.isfinite(y).all()
