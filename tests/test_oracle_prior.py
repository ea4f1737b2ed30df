"""Pins of the oracle's Ornstein-Uhlenbeck prior (Sec. 4.1.2, Eq. Minimised_functional).

* On equally spaced collinear pixels the exponential covariance is the AR(1)
  correlation rho^|i-j| (rho = exp(-dx/tau)), whose inverse is known in closed
  form: tridiagonal, 1/(1-rho^2) times diag(1, 1+rho^2, ..., 1+rho^2, 1) and
  off-diagonals -rho.  This pins the exponent, the distance scale and the solve.
* The distance is Euclidean: offsets (3, 4) and (5, 0) cells give equal entries
  (a Manhattan or Chebyshev distance would not).
* tau -> 0 makes Xi the identity: P = |z - eta|^2 / (2 sigma^2), dP = (z - eta) / sigma^2.
* dP/dz matches central differences of P; P >= 0 with P = 0 at z = eta.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def _ar1_inverse(m, rho):
    T = np.zeros((m, m))
    for i in range(m):
        T[i, i] = 1.0 if i in (0, m - 1) else 1.0 + rho * rho
        if i + 1 < m:
            T[i, i + 1] = T[i + 1, i] = -rho
    return T / (1.0 - rho * rho)


@pytest.mark.parametrize("m,dx,tau", [(7, 1e-4, 1.5e-3), (12, 4e-4, 1.5e-3), (5, 1e-3, 5e-4)])
def test_collinear_inverse_is_the_ar1_tridiagonal(m, dx, tau):
    from oracle.prior import OUPrior
    pr = OUPrior((1, m), dx, tau)
    v = np.random.default_rng(m).standard_normal((3, 1, m))
    T = _ar1_inverse(m, np.exp(-dx / tau))
    for j in range(3):
        np.testing.assert_allclose(pr.solve(v[j]).ravel(), T @ v[j].ravel(), rtol=1e-9, atol=1e-9)
    # a grid row of a 2-D grid is the same collinear set
    pr2 = OUPrior((4, m), dx, tau)
    row = slice(2 * m, 3 * m)
    np.testing.assert_allclose(np.linalg.inv(pr2.xi[row, row]), T, rtol=1e-8, atol=1e-8)


def test_distance_is_euclidean():
    from oracle.prior import OUPrior
    pr = OUPrior((6, 6), 1e-4, 3e-4)
    idx = lambda i, j: i * 6 + j
    a = pr.xi[idx(0, 0), idx(3, 4)]
    b = pr.xi[idx(0, 0), idx(0, 5)]
    c = pr.xi[idx(1, 1), idx(5, 4)]   # offset (4, 3)
    assert a == pytest.approx(b, rel=1e-12) and c == pytest.approx(b, rel=1e-12)
    assert pr.xi[idx(0, 0), idx(1, 1)] < pr.xi[idx(0, 0), idx(0, 1)]


def test_small_tau_reduces_to_independent_pixels():
    from oracle.prior import OUPrior
    pr = OUPrior((5, 5), 1e-4, 1e-7)
    z = np.random.default_rng(1).standard_normal((5, 5)) + 1500.0
    P, g = pr.term(z, 1500.0, 12.5)
    r = z - 1500.0
    assert P == pytest.approx(0.5 * np.sum(r * r) / 12.5 ** 2, rel=1e-12)
    np.testing.assert_allclose(g, r / 12.5 ** 2, rtol=1e-12)


def test_gradient_matches_central_differences():
    from oracle.prior import OUPrior
    pr = OUPrior((4, 5), 2e-4, 6e-4)
    rng = np.random.default_rng(3)
    z = 1500.0 + 20.0 * rng.standard_normal((4, 5))
    P, g = pr.term(z, 1490.0, 30.0)
    assert P > 0.0 and pr.term(np.full((4, 5), 1490.0), 1490.0, 30.0)[0] == 0.0
    h = 1e-3
    for i, j in [(0, 0), (1, 3), (3, 4), (2, 2)]:
        e = np.zeros_like(z)
        e[i, j] = h
        fd = (pr.term(z + e, 1490.0, 30.0)[0] - pr.term(z - e, 1490.0, 30.0)[0]) / (2 * h)
        assert fd == pytest.approx(g[i, j], rel=1e-6, abs=1e-12)


def test_prior_value_grad_sums_the_fields():
    from oracle.prior import OUPrior, prior_value_grad
    pr = OUPrior((4, 4), 1e-4, 2e-4)
    rng = np.random.default_rng(5)
    p0 = rng.uniform(0, 1, (3, 4, 4))
    c = 1500 + 10 * rng.standard_normal((4, 4))
    J, gp, gc = prior_value_grad(pr, p0, c, 0.5, 0.25, 1525.0, 62.5)
    parts = [pr.term(p0[k], 0.5, 0.25) for k in range(3)] + [pr.term(c, 1525.0, 62.5)]
    assert J == pytest.approx(sum(p[0] for p in parts), rel=1e-12)
    np.testing.assert_allclose(gp[1], parts[1][1], rtol=1e-12)
    np.testing.assert_allclose(gc, parts[3][1], rtol=1e-12)
