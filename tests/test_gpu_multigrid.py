"""Multigrid transfers and the data path without inverse crime, against the oracle.

Sec. 3.1 moves the parameters of a converged level to the next finer grid by
interpolation; Sec. 4.1.2 interpolates the measured data linearly to the time
grid of each level; Sec. 4.1.1 and Table 1 simulate the data on a grid finer
than every reconstruction level, with 236 point sensors on a square 0.2 mm
outside the target, and the bone phantom raises the upper speed bound to
3000 m/s (a smaller time step).  The tests run that path on the GPU (finer
data grid -> time interpolation -> level gradient) on a scaled-down copy of
the geometry and compare every stage with the oracle on the same inputs.
"""
import numpy as np
import pytest

import pat_synth as ps
from tests._problems import gpu_plan, oracle_grid, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("ns,nd,nb", [(32, 64, 2), (40, 58, 1), (64, 136, 3), (58, 40, 1)])
def test_prolong_matches_oracle(ns, nd, nb):
    from oracle.multigrid import prolong as o_prolong
    from paper_2505_08482_gb300.solver import prolong
    f = ps.rng_for(ns + nd).uniform(1400.0, 1650.0, size=(nb, ns, ns)).astype(np.float32)
    out = prolong(_dev(f), nd).cpu().numpy()
    ref = o_prolong(f.astype(np.float64), nd)
    assert np.max(np.abs(out - ref)) <= 2e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("nts,dts,dtd,ntd", [(1747, 12.1e-9, 19.2e-9, 1101), (400, 12.1e-9, 88.7e-9, 56),
                                             (300, 2e-8, 1e-8, 650)])
def test_time_interp_matches_oracle(nts, dts, dtd, ntd):
    from oracle.multigrid import time_interp as o_time_interp
    from paper_2505_08482_gb300.solver import time_interp
    y = ps.rng_for(nts).standard_normal((2, nts, 36)).astype(np.float32)
    out = time_interp(_dev(y), dts, dtd, ntd).cpu().numpy()
    ref = o_time_interp(y.astype(np.float64), dts, dtd, ntd)
    assert np.max(np.abs(out - ref)) <= 1e-5 * np.max(np.abs(ref))


def _level_params(n, L, U, T, c_bg=1430.0, dt=None):
    from oracle.grid import pml_auto
    dx = L / n
    dt = 0.3 * dx / U if dt is None else dt
    return dict(n=n, pml=pml_auto(n, 20), dx=dx, dt=dt, nt=int(round(T / dt)) + 1, c_ref=U, rho0=1000.0,
                pml_alpha=2.0, c_bg=c_bg)


@pytest.mark.parametrize("kind,U,level", [("circles", 1800.0, 40), ("water", 1800.0, 64), ("bone", 3000.0, 64)])
def test_fine_data_grid_to_level(kind, U, level):
    """Data on a finer grid (Ng 144) with the square 236-sensor geometry, time-interpolated to a
    coarser level, then the level's objective and gradient: each stage against the oracle."""
    from oracle.adjoint import adjoint_grad
    from oracle.forward import forward
    from oracle.multigrid import level_nt, prolong as o_prolong, time_interp as o_time_interp
    from oracle.sensors import sensor_matrix
    from paper_2505_08482_gb300.solver import time_interp
    L = ps.SIMPLE_L
    xy = ps.square_sensors()
    assert xy.shape == (236, 2)
    nd, K = 104, 4
    dx_d = L / nd
    dt_d = min(12.1e-9, 0.3 * dx_d / U)
    T = 4.8e-6
    gd = _level_params(nd, L, U, T, dt=dt_d)
    c_d, p0_d = ps.simple_phantom_c(kind, nd), ps.simple_phantom_p0(nd, K)
    plan_d = gpu_plan(gd, xy, K)
    assert plan_d.ng == 144
    y_d = plan_d.forward(_dev(c_d), _dev(p0_d)).cpu().numpy()
    og_d = oracle_grid(gd)
    y_ref = forward(og_d, c_d, p0_d, sensor_matrix(og_d, xy))
    assert rel_l2(y_d, y_ref) <= 1e-4
    ym = ps.add_noise(y_d.astype(np.float64), ps.rng_for(300))
    wts = ps.noise_weights(ym)
    # the level's time grid: dt_l = CFL dx_l / U, nt_l = round(T_data / dt_l) + 1
    gl = _level_params(level, L, U, (gd["nt"] - 1) * dt_d)
    assert gl["nt"] == level_nt((gd["nt"] - 1) * dt_d, gl["dt"])
    yl = time_interp(_dev(ym), dt_d, gl["dt"], gl["nt"])
    yl_ref = o_time_interp(ym.astype(np.float32).astype(np.float64), dt_d, gl["dt"], gl["nt"])
    assert rel_l2(yl.cpu().numpy(), yl_ref) <= 1e-6
    # level objective and gradient at a point between the start and the truth
    c_l = 0.5 * (o_prolong(c_d, level) + 1505.0)
    p0_l = 0.5 * o_prolong(p0_d, level)
    plan_l = gpu_plan(gl, xy, K)
    J, gp0, gc = plan_l.adjoint_grad(_dev(c_l), _dev(p0_l), yl, _dev(wts))
    og_l = oracle_grid(gl)
    Jo, gpo, gco = adjoint_grad(og_l, c_l, p0_l, sensor_matrix(og_l, xy), yl.cpu().numpy().astype(np.float64), wts)
    assert abs(J.item() - Jo) <= 1e-4 * Jo
    assert rel_l2(gp0.cpu().numpy(), gpo) <= 1e-3
    assert rel_l2(gc.cpu().numpy(), gco) <= 1e-3
