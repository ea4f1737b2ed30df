"""Pins of the oracle gradient: dot-product test (P4) and finite differences (P5)."""
import numpy as np
import pytest

from oracle import adjoint as A
from oracle import forward as F
from oracle.grid import Grid
from oracle.sensors import sensor_matrix
import pat_synth as ps


@pytest.mark.parametrize("alpha_max", [0.0, 2.0])
def test_p4_dot_product(alpha_max):
    rng = ps.rng_for(7)
    g = Grid(n=16, pml=8, dx=1e-4, dt=0.3e-4 / 1750.0, nt=40, c_ref=1750.0, alpha_max=alpha_max)
    S = sensor_matrix(g, ps.circle_sensors(16, 12, 1e-4))
    c = 1450.0 + 150.0 * rng.uniform(size=(16, 16))
    x = rng.standard_normal((2, 16, 16))
    r = rng.standard_normal((2, 40, 12))
    Ax = F.forward(g, c, x, S)
    ATr = A.adjoint_linear(g, c, S, r)
    lhs, rhs = np.sum(Ax * r), np.sum(x * ATr)
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(Ax) * np.linalg.norm(r)


def _problem(seed=3):
    w = ps.workload("tiny16", seed)
    rng = ps.rng_for(100 + seed)
    g = Grid(n=16, pml=8, dx=1e-4, dt=0.3e-4 / 1750.0, nt=60, c_ref=1750.0)
    S = sensor_matrix(g, w.sensors)
    ym = F.forward(g, w.c_true, w.p0_true, S) + 0.01 * rng.standard_normal((2, 60, 12))
    wt = np.array([3.0, 5.0])
    c0 = np.full((16, 16), 1520.0) + 10.0 * rng.standard_normal((16, 16))
    p00 = 0.7 * w.p0_true
    return g, S, ym, wt, c0, p00, rng


def test_p5_directional_finite_differences():
    g, S, ym, wt, c0, p00, rng = _problem()
    J, gp, gc = A.adjoint_grad(g, c0, p00, S, ym, wt)
    for _ in range(3):
        dp = rng.standard_normal(p00.shape)
        dc = rng.standard_normal(c0.shape)
        hp, hc = 1e-6, 1e-6 * 1500.0
        Jp = A.objective(g, c0 + hc * dc, p00 + hp * dp, S, ym, wt)[0]
        Jm = A.objective(g, c0 - hc * dc, p00 - hp * dp, S, ym, wt)[0]
        fd = 0.5 * (Jp - Jm)
        an = hp * np.sum(gp * dp) + hc * np.sum(gc * dc)
        assert abs(fd - an) <= 1e-7 * abs(an)
        Jp = A.objective(g, c0 + hc * dc, p00, S, ym, wt)[0]
        Jm = A.objective(g, c0 - hc * dc, p00, S, ym, wt)[0]
        assert abs(0.5 * (Jp - Jm) - hc * np.sum(gc * dc)) <= 1e-7 * abs(hc * np.sum(gc * dc))


def test_p5_individual_entries():
    g, S, ym, wt, c0, p00, rng = _problem(4)
    J, gp, gc = A.adjoint_grad(g, c0, p00, S, ym, wt)
    for (iy, ix) in ((8, 8), (3, 12), (0, 0), (15, 7)):
        h = 1e-6 * 1500.0
        cp, cm = c0.copy(), c0.copy()
        cp[iy, ix] += h
        cm[iy, ix] -= h
        fd = (A.objective(g, cp, p00, S, ym, wt)[0] - A.objective(g, cm, p00, S, ym, wt)[0]) / (2 * h)
        assert abs(fd - gc[iy, ix]) <= 1e-6 * np.abs(gc).max()
        h = 1e-6
        pp, pm = p00.copy(), p00.copy()
        pp[1, iy, ix] += h
        pm[1, iy, ix] -= h
        fd = (A.objective(g, c0, pp, S, ym, wt)[0] - A.objective(g, c0, pm, S, ym, wt)[0]) / (2 * h)
        assert abs(fd - gp[1, iy, ix]) <= 1e-6 * np.abs(gp).max()


def test_single_sample_gradient_is_sensor_transpose():
    # Nt = 1: y = S p0, so dJ/dp0 = S^T w (S p0 - y) and dJ/dc = 0
    rng = ps.rng_for(5)
    g = Grid(n=16, pml=8, dx=1e-4, dt=0.3e-4 / 1750.0, nt=1, c_ref=1750.0)
    S = sensor_matrix(g, ps.circle_sensors(16, 12, 1e-4))
    p0 = rng.uniform(size=(1, 16, 16))
    c = 1500.0 + 50 * rng.uniform(size=(16, 16))
    ym = rng.standard_normal((1, 1, 12))
    J, gp, gc = A.adjoint_grad(g, c, p0, S, ym, [2.0])
    r = 2.0 * (S @ g.pad(p0[0]).ravel() - ym[0, 0])
    assert np.abs(gp[0] - g.crop((S.T @ r).reshape(g.ng, g.ng))).max() <= 1e-15 * np.abs(gp).max()
    assert np.abs(gc).max() == 0.0


def test_gradient_vanishes_at_noise_free_truth():
    w = ps.workload("tiny16", 2)
    g = Grid(n=16, pml=8, dx=1e-4, dt=0.3e-4 / 1750.0, nt=50, c_ref=1750.0)
    S = sensor_matrix(g, w.sensors)
    y = F.forward(g, w.c_true, w.p0_true, S)
    J, gp, gc = A.adjoint_grad(g, w.c_true, w.p0_true, S, y, [1.0, 1.0])
    assert J == 0.0 and np.abs(gp).max() == 0.0 and np.abs(gc).max() == 0.0
