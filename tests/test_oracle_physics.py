"""Pins of the oracle forward solve against closed forms of the physics.

* P1: homogeneous c = c_ref, no PML, periodic grid: the k-space leapfrog is
  exact in time, p^n = F^-1[cos(c |k| n dt) F p0], at any CFL.
* P2: a Gaussian p0 in free 2-D space has p(r,t) = A s^2 int_0^inf
  exp(-k^2 s^2/2) cos(c k t) J0(k r) k dk; compared before any periodic image
  arrives.
* 1-D interface: a plane pulse crossing c1 -> c2 (uniform density) is
  transmitted with 2 c2/(c1+c2) and reflected with (c2-c1)/(c2+c1).
* PML: a plane pulse crossing the two absorbing layers keeps exp(-int alpha/c dx)
  of its amplitude (each field decays at the rate alpha inside the layer).
"""
import numpy as np
import pytest
from scipy.special import j0

from oracle import forward as F
from oracle.grid import Grid, make_grid, pml_auto, time_step
import pat_synth as ps


@pytest.mark.parametrize("cfl", [0.3, 0.9])
def test_p1_homogeneous_exact_in_time(cfl):
    n, c = 24, 1500.0
    g = Grid(n=n, pml=4, dx=1e-4, dt=cfl * 1e-4 / c, nt=2, c_ref=c, alpha_max=0.0)
    p0 = g.pad(ps.rng_for(1).standard_normal((n, n)))
    fields = F.pressure_fields(g, g.medium(np.full((n, n), c)), p0, 30)
    kabs = np.sqrt(g.KX ** 2 + g.KY ** 2)
    for n_ in (1, 2, 7, 30):
        exact = np.real(np.fft.ifft2(np.cos(c * kabs * n_ * g.dt) * np.fft.fft2(p0)))
        assert np.abs(fields[n_] - exact).max() <= 1e-12 * np.abs(exact).max()


def test_p1_fails_for_wrong_reference_speed():
    # kappa must use the medium speed for exactness; a mismatch is detectable
    n, c = 24, 1500.0
    g = Grid(n=n, pml=4, dx=1e-4, dt=0.3e-4 / c, nt=2, c_ref=1.2 * c, alpha_max=0.0)
    p0 = g.pad(ps.rng_for(1).standard_normal((n, n)))
    fields = F.pressure_fields(g, g.medium(np.full((n, n), c)), p0, 10)
    kabs = np.sqrt(g.KX ** 2 + g.KY ** 2)
    exact = np.real(np.fft.ifft2(np.cos(c * kabs * 10 * g.dt) * np.fft.fft2(p0)))
    assert np.abs(fields[10] - exact).max() > 1e-6 * np.abs(exact).max()


def test_p2_gaussian_free_space_closed_form():
    dx, c, ng = 1e-4, 1500.0, 256
    g = Grid(n=ng, pml=0, dx=dx, dt=0.3 * dx / c, nt=2, c_ref=c, alpha_max=0.0)
    s = 3 * dx
    x = (np.arange(ng) - ng // 2) * dx
    X, Y = np.meshgrid(x, x)
    p0 = np.exp(-(X ** 2 + Y ** 2) / (2 * s * s))
    nsteps = 333                      # c t = 100 cells; nearest image is 256 cells away
    p = F.pressure_fields(g, g.medium(np.full((ng, ng), c)), p0, nsteps)[-1]
    t = nsteps * g.dt
    k = np.linspace(0.0, 12.0 / s, 400001)
    r = np.abs(x[ng // 2: ng // 2 + 90])
    exact = np.array([s * s * np.trapezoid(np.exp(-k * k * s * s / 2) * np.cos(c * k * t) * j0(k * rr) * k, k)
                      for rr in r])
    num = p[ng // 2, ng // 2: ng // 2 + 90]
    assert np.abs(num - exact).max() <= 1e-6 * np.abs(exact).max()


def test_interface_reflection_and_transmission():
    dx, n = 1e-4, 400
    c1, c2 = 1500.0, 1800.0
    g = Grid(n=n, pml=0, dx=dx, dt=0.3 * dx / c2, nt=2, c_ref=c2, alpha_max=0.0)
    cx = np.where(np.arange(n) < 250, c1, c2)
    cd = np.broadcast_to(cx[None, :], (n, n)).copy()
    xs = np.arange(n)
    p0 = np.broadcast_to(np.exp(-(xs - 150.0) ** 2 / 32.0)[None, :], (n, n)).copy()
    nsteps = int(round(160 * dx / c1 / g.dt))
    row = F.pressure_fields(g, cd, p0, nsteps)[-1][0]
    R = (c2 - c1) / (c2 + c1)
    trans = row[280:370].max()
    refl = row[170:215][np.argmax(np.abs(row[170:215]))]
    assert abs(trans / (0.5 * (1 + R)) - 1) < 2e-3
    assert abs(refl / (0.5 * R) - 1) < 2e-2


def test_pml_transmission_matches_absorption_integral():
    dx, c, n, P, am = 1e-4, 1500.0, 100, 20, 0.1
    g = Grid(n=n, pml=P, dx=dx, dt=0.3 * dx / c, nt=2, c_ref=c, alpha_max=am)
    ng = g.ng
    g.ay = np.ones_like(g.ay)      # plane wave along x: absorb along x only
    g.asy = np.ones_like(g.asy)
    xs = np.arange(ng)
    x0, D = ng // 2, 30
    p0 = np.broadcast_to(np.exp(-(xs - x0) ** 2 / 18.0)[None, :], (ng, ng)).copy()
    nsteps = int(round((ng - D) / 0.3))
    row = F.pressure_fields(g, g.medium(np.full((n, n), c)), p0, nsteps)[-1][ng // 2]
    # the right-going half pulse crossed the right layer (depth 0 -> P+1 at the
    # periodic seam) and the left layer (depth P -> 0)
    s = np.linspace(0.0, 1.0, 200001)
    prof = lambda xi: am * (c / dx) * (xi / P) ** 4
    path = np.trapezoid(prof(s * (P + 1)), s) * (P + 1) + np.trapezoid(prof(s * P), s) * P
    expect = 0.5 * np.exp(-path * dx / c)
    got = row[x0 - D - 15: x0 - D + 15].max()
    assert abs(got / expect - 1) < 2e-2


def test_time_step_and_pml_rules():
    assert time_step(1e-4, 0.3, 1750.0) == pytest.approx(0.3e-4 / 1750.0, rel=1e-15)
    g = make_grid(64, 1e-4, 10, c_ref=1750.0)
    assert g.pml == pml_auto(64) and g.ng == 108
    # interior cells are not absorbed, the outermost layer cell is
    assert np.all(g.a_cell[g.pml:g.pml + g.n] == 1.0)
    assert g.a_cell[0] < g.a_cell[g.pml - 1] < 1.0
