"""Cluster-resident stepping (one 16-CTA thread-block cluster per data set, wavefield on chip,
row and column spectra exchanged through distributed shared memory) against the oracle and
the launched passes, on the 256 x 256 domain (Ng 300, the side it is compiled for).

The forward traces must match the oracle to 1e-4 and the launched passes to FP32 rounding;
a gradient whose forward sweep and segment recomputes run cluster-resident (checkpoints every
7 steps: ragged segments restored from checkpoints) must match the oracle's gradient to 1e-3;
more data sets than the GPU runs clusters at once still give the same traces.
"""
import numpy as np
import pytest

import pat_synth as ps
from tests._problems import grid_params, oracle_grid, gpu_plan, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _case(K, M, seed):
    n = 256
    rng = ps.rng_for(seed)
    c = ps.ellipse_phantom(n, 4, rng)
    p0 = np.stack([ps.vessel_p0(n, rng) for _ in range(K)])
    xy = ps.circle_sensors(n, M, 1e-4, phase=0.2)
    return n, c, p0, xy


def test_cluster_forward_matches_oracle_and_launched_passes():
    from oracle.forward import forward
    from oracle.sensors import sensor_matrix
    n, c, p0, xy = _case(2, 32, 31)
    gp = grid_params(n, 60)
    g = oracle_grid(gp)
    ref = forward(g, c, p0, sensor_matrix(g, xy))
    plan = gpu_plan(gp, xy, 2)
    assert plan.ng == 300 and plan.cluster_capacity >= 1
    y_l = plan.forward(_dev(c), _dev(p0)).cpu().numpy()
    plan.cluster = True
    assert plan.cluster
    y_c = plan.forward(_dev(c), _dev(p0)).cpu().numpy()
    assert rel_l2(y_c, ref) <= 1e-4, rel_l2(y_c, ref)
    assert rel_l2(y_c, y_l) <= 1e-5, rel_l2(y_c, y_l)
    plan.cluster = False
    assert not plan.cluster


def test_cluster_gradient_matches_oracle():
    from oracle.adjoint import adjoint_grad
    from oracle.forward import forward
    from oracle.sensors import sensor_matrix
    n, c, p0, xy = _case(2, 24, 32)
    gp = grid_params(n, 50)
    g = oracle_grid(gp)
    S = sensor_matrix(g, xy)
    ym = ps.add_noise(forward(g, c, p0, S), ps.rng_for(5))
    wt = np.array([1.0, 2.0])
    c0 = np.full((n, n), 1520.0)
    J, gp0, gc = adjoint_grad(g, c0, 0.5 * p0, S, ym, wt)
    plan = gpu_plan(gp, xy, 2, ckpt_every=7)
    plan.cluster = True
    Jg, a, b = plan.adjoint_grad(_dev(c0), _dev(0.5 * p0), _dev(ym), _dev(wt))
    assert abs(Jg.item() - J) <= 1e-4 * J
    assert rel_l2(a.cpu().numpy(), gp0) <= 1e-3, rel_l2(a.cpu().numpy(), gp0)
    assert rel_l2(b.cpu().numpy(), gc) <= 1e-3, rel_l2(b.cpu().numpy(), gc)


def test_more_data_sets_than_resident_clusters():
    n, c, _, xy = _case(1, 16, 33)
    gp = grid_params(n, 24)
    plan1 = gpu_plan(gp, xy, 1)
    K = plan1.cluster_capacity + 1
    rng = ps.rng_for(34)
    p0 = np.stack([ps.vessel_p0(n, rng) for _ in range(K)])
    plan = gpu_plan(gp, xy, K)
    y_l = plan.forward(_dev(c), _dev(p0)).cpu().numpy()
    plan.cluster = True
    y_c = plan.forward(_dev(c), _dev(p0)).cpu().numpy()
    assert rel_l2(y_c, y_l) <= 1e-5, rel_l2(y_c, y_l)


def test_cluster_form_only_on_its_grid_side():
    from paper_2505_08482_gb300 import _binding as B
    plan = gpu_plan(grid_params(128, 10), ps.circle_sensors(128, 8, 1e-4), 1)   # Ng 180
    assert plan.cluster_capacity == 0
    with pytest.raises(B.PatError):
        plan.cluster = True


def test_cluster_batched_plan_matches_launched_passes():
    """Two instances with their own c in one batched plan (the medium of each data set is its
    instance's): the cluster-resident sweep and gradient equal the launched passes'."""
    n = 256
    rng = ps.rng_for(36)
    cs = np.stack([ps.ellipse_phantom(n, 3, rng), ps.ellipse_phantom(n, 5, rng)])
    Ks = [1, 2]
    p0 = np.stack([ps.vessel_p0(n, rng) for _ in range(sum(Ks))])
    xy = ps.circle_sensors(n, 16, 1e-4, phase=0.4)
    gp = grid_params(n, 40)
    plan = gpu_plan(gp, xy, Ks, ckpt_every=9)
    y_l = plan.forward(_dev(cs), _dev(p0)).cpu().numpy()
    ym = _dev(y_l * 1.01 + 0.001)
    wt = _dev(np.array([1.0, 0.5, 2.0]))
    c0 = _dev(np.full((2, n, n), 1510.0))
    J_l, a_l, b_l = [t.cpu().numpy() for t in plan.adjoint_grad(c0, _dev(0.5 * p0), ym, wt)]
    plan.cluster = True
    y_c = plan.forward(_dev(cs), _dev(p0)).cpu().numpy()
    J_c, a_c, b_c = [t.cpu().numpy() for t in plan.adjoint_grad(c0, _dev(0.5 * p0), ym, wt)]
    assert rel_l2(y_c, y_l) <= 1e-5
    assert np.all(np.abs(J_c - J_l) <= 1e-5 * np.abs(J_l))
    assert rel_l2(a_c, a_l) <= 1e-4 and rel_l2(b_c, b_l) <= 1e-4
