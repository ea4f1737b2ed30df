"""Batched solves: several instances in one plan, graphs, autotuner, batched reconstruction.

A batched plan runs every pass once for all instances; each data set uses its
own instance's c, and the per-instance J and dJ/dc are reduced in the same
order as for a plan of that instance alone, so the results must be identical.
"""
import numpy as np
import pytest

import pat_synth as ps
from tests._problems import grid_params, gpu_plan, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _instances(n, Ks, nt, seed=0):
    rng = ps.rng_for(seed)
    out = []
    for K in Ks:
        c = ps.ellipse_phantom(n, 3, rng)
        p0 = np.stack([ps.blob_p0(n, 3, rng, sigma_cells=(1.5, 3.0)) for _ in range(K)])
        out.append((c, p0))
    return out


@pytest.mark.parametrize("n,variant", [(40, None), (64, 0), (64, 3)])
def test_batched_plan_equals_single_plans(n, variant):
    Ks = [1, 3, 2]
    xy = ps.circle_sensors(n, 16, 1e-4)
    gp = grid_params(n, 90)
    inst = _instances(n, Ks, 90)
    bplan = gpu_plan(gp, xy, Ks, ckpt_every=16)
    if variant is not None:
        bplan.variant = variant
    c_b = _dev(np.stack([c for c, _ in inst]))
    p0_b = _dev(np.concatenate([p for _, p in inst]))
    yb = bplan.forward(c_b, p0_b)
    rng = ps.rng_for(4)
    ym = _dev(yb.cpu().numpy() + 0.01 * rng.standard_normal(yb.shape))
    w = _dev(rng.uniform(0.5, 2.0, size=sum(Ks)))
    c0 = _dev(np.stack([np.full((n, n), 1490.0 + 10 * i) for i in range(len(Ks))]))
    Jb, gpb, gcb = bplan.adjoint_grad(c0, 0.5 * p0_b, ym, w)
    k0 = 0
    for i, (c, p0) in enumerate(inst):
        K = Ks[i]
        plan = gpu_plan(gp, xy, K, ckpt_every=16)
        if variant is not None:
            plan.variant = variant
        y = plan.forward(_dev(c), _dev(p0))
        assert torch.equal(y, yb[k0:k0 + K])
        J, gp0, gc = plan.adjoint_grad(c0[i].contiguous(), (0.5 * p0_b[k0:k0 + K]).contiguous(),
                                       ym[k0:k0 + K].contiguous(), w[k0:k0 + K].contiguous())
        assert J.item() == Jb[i].item()
        assert torch.equal(gp0, gpb[k0:k0 + K]) and torch.equal(gc, gcb[i])
        k0 += K


def test_graph_replay_equals_direct_calls():
    n = 64
    xy = ps.circle_sensors(n, 24, 1e-4)
    gp = grid_params(n, 120)
    (c, p0), = _instances(n, [2], 120, seed=3)
    plan = gpu_plan(gp, xy, 2, ckpt_every=32)
    cd, pd = _dev(c), _dev(p0)
    ym = _dev(ps.rng_for(1).standard_normal((2, 120, 24)) * 0.05)
    w = _dev(np.array([1.0, 3.0]))
    y_ref = plan.forward(cd, pd).clone()
    J_ref, g_ref, c_ref = [t.clone() for t in plan.adjoint_grad(cd, pd, ym, w)]
    # the reference calls used the plan's workspaces on the default stream: the replays on
    # another stream share them and must not start before those calls end
    torch.cuda.synchronize()
    plan.set_graphs(True)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        y = torch.empty_like(y_ref)
        gp0 = torch.empty_like(g_ref)
        gc = torch.empty_like(c_ref)
        J = torch.empty_like(J_ref)
        for _ in range(3):    # capture, then two replays
            plan.forward(cd, pd, y=y, stream=stream)
            plan.adjoint_grad(cd, pd, ym, w, grad_p0=gp0, grad_c=gc, J=J, stream=stream)
            stream.synchronize()
            assert torch.equal(y, y_ref) and torch.equal(gp0, g_ref) and torch.equal(gc, c_ref)
            assert J.item() == J_ref.item()
    plan.set_graphs(False)


def test_graph_cache_is_bounded_and_recaptures_evicted_calls():
    """20 output buffers give 20 keys: the plan keeps 16 graphs, a call whose graph was
    dropped is captured again, and every replay equals the direct call."""
    n = 40
    xy = ps.circle_sensors(n, 12, 1e-4)
    gp = grid_params(n, 60)
    (c, p0), = _instances(n, [1], 60, seed=5)
    plan = gpu_plan(gp, xy, 1, ckpt_every=16)
    cd, pd = _dev(c), _dev(p0)
    y_ref = plan.forward(cd, pd).clone()
    torch.cuda.synchronize()   # the replays on another stream share the plan's workspace
    plan.set_graphs(True)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ys = [torch.full_like(y_ref, float("nan")) for _ in range(20)]
        for rep in range(2):    # captures (with evictions), then recaptures of the dropped ones
            for y in ys:
                plan.forward(cd, pd, y=y, stream=stream)
            stream.synchronize()
            for y in ys:
                assert torch.equal(y, y_ref)
                y.fill_(float("nan"))
    plan.set_graphs(False)


def test_autotune_selects_a_variant_with_identical_physics():
    n = 128
    xy = ps.circle_sensors(n, 32, 1e-4)
    gp = grid_params(n, 60)
    (c, p0), = _instances(n, [4], 60, seed=2)
    plan = gpu_plan(gp, xy, 4)
    for gradient in (False, True):   # forward steps, then whole gradient evaluations
        ms = plan.autotune(gradient=gradient)
        assert set(ms) == set(range(-1, plan.variants)) and all(v > 0 for v in ms.values())
        assert plan.variant == min(ms, key=ms.get)
    y = plan.forward(_dev(c), _dev(p0)).cpu().numpy()
    plan.variant = -1
    assert rel_l2(y, plan.forward(_dev(c), _dev(p0)).cpu().numpy()) <= 1e-5


@pytest.mark.parametrize("with_prior", [False, True])
def test_batched_reconstruction_equals_single_reconstructions(with_prior):
    from oracle.forward import forward
    from oracle.sensors import sensor_matrix
    from tests._problems import oracle_grid
    from paper_2505_08482_gb300.solver import ReconConfig, reconstruct, reconstruct_batched
    n = 64
    xy = ps.circle_sensors(n, 32, 1e-4)
    gp = grid_params(n, 200)
    g = oracle_grid(gp)
    S = sensor_matrix(g, xy)
    insts = []
    for i, (c, p0) in enumerate(_instances(n, [1, 2, 1], 200, seed=7)):
        y = ps.add_noise(forward(g, c, p0, S), ps.rng_for(20 + i))
        insts.append(dict(y_meas=_dev(y), w=_dev(ps.noise_weights(y)), c_init=_dev(np.full((n, n), 1510.0))))
    cfg = ReconConfig(levels=(32, 64), L=n * 1e-4, dt_data=g.dt, nt_data=g.nt, sensors_xy=xy, K=1, iters=4,
                      mem=5, ckpt_every=32)
    if with_prior:   # Ornstein-Uhlenbeck terms: each instance's solves must not see the others'
        cfg.prior_tau, cfg.prior_eta_c, cfg.prior_sigma_c = 1.5e-3, 1510.0, 50.0
        cfg.prior_eta_p0, cfg.prior_sigma_p0 = 0.5, 0.25
    res, ms = reconstruct_batched(cfg, insts)
    for ins, (c_b, p0_b, rows_b, st_b) in zip(insts, res):
        cfg.K = int(ins["y_meas"].shape[0])
        c_s, p0_s, rows_s, st_s, _ = reconstruct(cfg, ins["y_meas"], ins["w"], ins["c_init"])
        assert st_b == st_s and len(rows_b) == len(rows_s)
        for a, b in zip(rows_b, rows_s):
            assert (a["level"], a["it"], a["alpha"], a["trials"]) == (b["level"], b["it"], b["alpha"], b["trials"])
            assert a["J"] == b["J"] and a["J_new"] == b["J_new"]
        assert torch.equal(c_b, c_s) and torch.equal(p0_b, p0_s)


def test_tracked_errors_and_joint_targets():
    """E_c and E_p0 (Eq. RelativeError) reported per iteration equal the host's values at the
    returned point, and an instance with both targets leaves a level once it meets both."""
    from oracle.forward import forward
    from oracle.metrics import relative_error
    from oracle.sensors import sensor_matrix
    from tests._problems import oracle_grid
    from paper_2505_08482_gb300.solver import ReconConfig, reconstruct_batched
    n = 64
    xy = ps.circle_sensors(n, 32, 1e-4)
    gp = grid_params(n, 200)
    g = oracle_grid(gp)
    S = sensor_matrix(g, xy)
    (c, p0), = _instances(n, [2], 200, seed=11)
    y = ps.add_noise(forward(g, c, p0, S), ps.rng_for(33))
    base = dict(y_meas=_dev(y), w=_dev(ps.noise_weights(y)), c_init=_dev(np.full((n, n), 1510.0)),
                c_true=_dev(c), p0_true=_dev(p0))
    cfg = ReconConfig(levels=(32, 64), L=n * 1e-4, dt_data=g.dt, nt_data=g.nt, sensors_xy=xy, K=2, iters=4, mem=5)
    (c_r, p0_r, rows, st), = reconstruct_batched(cfg, [base])[0]
    last = rows[-1]
    assert last["level"] == 1
    assert abs(last["Ec"] - relative_error(c, c_r.cpu().numpy())) <= 1e-3 * last["Ec"]
    ep_host = 100.0 * np.linalg.norm(p0_r.cpu().numpy() - p0) / np.linalg.norm(p0)
    assert abs(last["Ep0"] - ep_host) <= 1e-3 * ep_host
    # targets met at once: one iteration per level; a target for p0 alone that is never met: all iterations
    (_, _, rows_easy, _), = reconstruct_batched(cfg, [dict(base, ec_target=1e3, ep0_target=1e3)])[0]
    assert [r["level"] for r in rows_easy] == [0, 1]
    (_, _, rows_hard, _), = reconstruct_batched(cfg, [dict(base, ec_target=1e3, ep0_target=1e-6)])[0]
    assert len(rows_hard) == len(rows)
