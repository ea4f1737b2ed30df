"""Invariants of the oracle: energy (P3), linearity (P6), exactness of interpolants."""
import numpy as np
import pytest

from oracle import forward as F
from oracle.grid import Grid
from oracle.multigrid import prolong, time_interp
from oracle.sensors import sensor_matrix
import pat_synth as ps


def test_p3_energy_conserved_without_pml():
    n = 24
    g = Grid(n=n, pml=4, dx=1e-4, dt=0.3e-4 / 1750.0, nt=2, c_ref=1750.0, alpha_max=0.0)
    rng = ps.rng_for(2)
    p0 = g.pad(rng.standard_normal((n, n)))
    c = g.medium(1400.0 + 300.0 * rng.uniform(size=(n, n)))
    E = F.energy_history(g, c, p0, 80)
    assert np.abs(E - E[0]).max() <= 1e-12 * abs(E[0])


def test_p3_energy_decays_with_pml():
    w = ps.workload("plain64", 0)
    g = Grid(n=64, pml=22, dx=1e-4, dt=0.3e-4 / 1750.0, nt=2, c_ref=1750.0)
    E = F.energy_history(g, g.medium(w.c_true), g.pad(w.p0_true[0]), 400)
    assert E[-1] < 0.2 * E[0]
    assert np.all(np.diff(E[200:]) <= 1e-12 * E[0])


def test_p6_linearity_in_p0():
    w = ps.workload("tiny16", 1)
    g = Grid(n=16, pml=8, dx=1e-4, dt=0.3e-4 / 1750.0, nt=30, c_ref=1750.0)
    S = sensor_matrix(g, w.sensors)
    y1 = F.forward(g, w.c_true, w.p0_true, S)
    y2 = F.forward(g, w.c_true, -2.5 * w.p0_true, S)
    assert np.abs(y2 + 2.5 * y1).max() <= 1e-12 * np.abs(y1).max()
    ysum = F.forward(g, w.c_true, w.p0_true[:1] + w.p0_true[1:], S)
    assert np.abs(ysum[0] - y1[0] - y1[1]).max() <= 1e-12 * np.abs(y1).max()


def test_sensor_bilinear_exact_on_affine_fields():
    g = Grid(n=32, pml=20, dx=2e-4, dt=1e-8, nt=2, c_ref=1750.0)
    xy = ps.circle_sensors(32, 40, 2e-4, radius_cells=14.3, phase=0.1)
    S = sensor_matrix(g, xy)
    gi = np.arange(g.ng)
    # physical coordinate of grid cell centres in the domain frame
    X = ((gi - g.pml + 0.5) * g.dx)[None, :] + 0 * gi[:, None]
    Y = ((gi - g.pml + 0.5) * g.dx)[:, None] + 0 * gi[None, :]
    f = 0.3 + 170.0 * X - 420.0 * Y
    got = S @ f.ravel()
    assert np.allclose(got, 0.3 + 170.0 * xy[:, 0] - 420.0 * xy[:, 1], rtol=0, atol=1e-12)
    assert np.allclose(np.asarray(S.sum(axis=1)).ravel(), 1.0, atol=1e-15)


def test_prolongation_exact_on_affine_interior_and_constants():
    nc, nf = 16, 32
    t = lambda n: (np.arange(n) + 0.5) / n      # cell centres of the unit domain
    Xc, Yc = np.meshgrid(t(nc), t(nc))
    Xf, Yf = np.meshgrid(t(nf), t(nf))
    f = prolong(2.0 - 3.0 * Xc + 5.0 * Yc, nf)
    ref = 2.0 - 3.0 * Xf + 5.0 * Yf
    inner = slice(1, nf - 1)
    assert np.abs(f[inner, inner] - ref[inner, inner]).max() < 1e-13
    assert np.abs(prolong(np.full((3, nc, nc), 7.25), nf) - 7.25).max() == 0.0


def test_time_interp_exact_on_linear_signals():
    dt_s, dt_d = 1e-8, 2.7e-8
    t = np.arange(300) * dt_s
    y = np.stack([np.stack([1.0 + 3e7 * t, -2.0 + 1e6 * t], axis=1)])
    out = time_interp(y, dt_s, dt_d, 100)
    td = np.arange(100) * dt_d
    assert np.abs(out[0, :, 0] - (1.0 + 3e7 * td)).max() < 1e-12
    assert np.abs(out[0, :, 1] - (-2.0 + 1e6 * td)).max() < 1e-12


def test_relative_error_values_of_eq_relative_error():
    """Eq. (RelativeError): 100 % ||true - rec|| / ||true||, the Euclidean norm over all cells."""
    from oracle.metrics import relative_error
    rng = ps.rng_for(4)
    true = 1500.0 + 40.0 * rng.standard_normal((12, 12))
    assert relative_error(true, true) == 0.0
    assert relative_error(true, 0.97 * true) == pytest.approx(3.0, rel=1e-12)
    assert relative_error(true, np.zeros_like(true)) == pytest.approx(100.0, rel=1e-12)
    # an error orthogonal to the true field adds in quadrature: 3-4-5 on two cells
    t2 = np.array([[4.0, 0.0]])
    assert relative_error(t2, np.array([[4.0, 3.0]])) == pytest.approx(75.0, rel=1e-12)
    # a norm over cells, not a mean of per-cell ratios: one wrong cell of two
    assert relative_error(np.array([1.0, 10.0]), np.array([0.0, 10.0])) == pytest.approx(
        100.0 / np.sqrt(101.0), rel=1e-12)
