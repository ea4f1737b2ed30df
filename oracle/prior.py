"""Ornstein-Uhlenbeck prior of the objective (oracle, FP64).

Test infrastructure: only tests/, the smoke check and the benchmark's CPU
baseline import this package.

Eq. (Minimised_functional) adds, for the speed of sound and for every initial
pressure, the regularising term 1/2 || L_z (z - eta_z) ||^2 with
L_z^T L_z = Gamma_z^{-1}.  Sec. 4.1.2 gives the Ornstein-Uhlenbeck covariance
Gamma_z = sigma_z^2 Xi with Xi_ij = exp(-||r_i - r_j|| / tau), r_i the pixel
locations and tau the characteristic length.  So the term is
    P(z) = 1/2 (z - eta)^T Xi^{-1} (z - eta) / sigma^2,
    dP/dz = Xi^{-1} (z - eta) / sigma^2.
Here Xi is built densely from that definition and factorised by Cholesky (it
is symmetric positive definite); this is only practical for small grids.

Readings: r_i are the cell centres of the reconstruction grid (the offset
cancels in the distances); the term uses the grid of the current multigrid
level, i.e. the pixel spacing of that level with tau fixed in metres.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def pixel_points(shape, dx: float):
    """Cell centres (x, y) of a grid of shape (rows, cols) with spacing dx, row-major."""
    ny, nx = shape
    yy, xx = np.meshgrid((np.arange(ny) + 0.5) * dx, (np.arange(nx) + 0.5) * dx, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel()], axis=1)


def unit_covariance(points, tau: float, rows=None):
    """Xi_ij = exp(-||r_i - r_j|| / tau) (Sec. 4.1.2); rows: only those rows i (index array)."""
    a = points if rows is None else points[np.asarray(rows)]
    d = np.sqrt(((a[:, None, :] - points[None, :, :]) ** 2).sum(-1))
    return np.exp(-d / tau)


class OUPrior:
    """Xi of one grid, factorised once; solve(v) = Xi^{-1} v for fields of that grid."""

    def __init__(self, shape, dx: float, tau: float):
        self.shape = tuple(shape)
        self.xi = unit_covariance(pixel_points(self.shape, dx), tau)
        self.cho = sla.cho_factor(self.xi, lower=True)

    def solve(self, v):
        v = np.asarray(v, dtype=np.float64)
        flat = v.reshape(-1, self.xi.shape[0]).T
        return sla.cho_solve(self.cho, flat).T.reshape(v.shape)

    def term(self, z, eta: float, sigma: float):
        """(P, dP/dz) of one field z for mean eta and standard deviation sigma."""
        r = np.asarray(z, dtype=np.float64) - eta
        s = self.solve(r)
        return 0.5 * float(np.sum(r * s)) / sigma ** 2, s / sigma ** 2


def prior_value_grad(prior: OUPrior, p0, c, eta_p0: float, sigma_p0: float, eta_c: float, sigma_c: float):
    """Prior part of the objective for p0[K][n][n] and c[n][n]: (value, dP/dp0, dP/dc)."""
    J = 0.0
    gp = np.empty(np.shape(p0))
    for k in range(np.shape(p0)[0]):
        v, gp[k] = prior.term(p0[k], eta_p0, sigma_p0)
        J += v
    v, gc = prior.term(c, eta_c, sigma_c)
    return J + v, gp, gc
