"""Coarse-to-fine multigrid schedule (oracle, FP64).

Sec. 3.1: start on a coarse discretisation, iterate until converged, linearly
interpolate the parameters to the next finer grid as its initial guess, and
repeat up to the finest grid.  Sec. 4.1.2: the measured data is linearly
interpolated to the time grid of each level, and every level keeps the same
physical domain.

Readings: every level covers the same L x L domain with dx_l = L / N_l,
dt_l = CFL dx_l / c_ref and Nt_l = round(T / dt_l) + 1 with T = (Nt-1) dt of
the data (this reproduces the N_t column of Table 1 from its Delta t column);
the PML is the smallest width >= 20 cells with a 5-smooth, even grid;
prolongation is bilinear on cell-centred physical coordinates with constant
extension beyond the outermost coarse cell centres; data past the last sample
are held constant.  The L-BFGS memory restarts on every level.
"""
from __future__ import annotations

import numpy as np

from .adjoint import adjoint_grad, objective
from .grid import make_grid
from .lbfgs import projected_lbfgs
from .prior import OUPrior, prior_value_grad
from .sensors import sensor_matrix


def level_nt(T: float, dt: float) -> int:
    """Number of time samples on a level: round(T / dt) + 1."""
    return int(round(T / dt)) + 1


def time_interp(y, dt_src: float, dt_dst: float, nt_dst: int):
    """Linear interpolation of y[K][Nt_src][M] (t = n dt_src) to t = n dt_dst."""
    y = np.asarray(y, dtype=np.float64)
    K, nt_src, M = y.shape
    t_src = np.arange(nt_src) * dt_src
    t_dst = np.arange(nt_dst) * dt_dst
    out = np.empty((K, nt_dst, M))
    for k in range(K):
        for m in range(M):
            out[k, :, m] = np.interp(t_dst, t_src, y[k, :, m])
    return out


def _interp_weights(n_src: int, n_dst: int):
    """Index/weight pairs mapping n_dst cell centres onto n_src cell centres (same extent)."""
    u = (np.arange(n_dst) + 0.5) * (n_src / n_dst) - 0.5
    u = np.clip(u, 0.0, n_src - 1.0)
    i0 = np.minimum(np.floor(u).astype(int), max(n_src - 2, 0))
    f = u - i0
    i1 = np.minimum(i0 + 1, n_src - 1)
    return i0, i1, f


def prolong(f, n_dst: int):
    """Bilinear interpolation of f[..][n][n] to [..][n_dst][n_dst] (same physical domain)."""
    f = np.asarray(f, dtype=np.float64)
    n_src = f.shape[-1]
    i0, i1, fx = _interp_weights(n_src, n_dst)
    rows = f[..., i0, :] * (1.0 - fx)[:, None] + f[..., i1, :] * fx[:, None]
    return rows[..., i0] * (1.0 - fx) + rows[..., i1] * fx


def reconstruct(levels, L, T, sensors_xy, y_meas, dt_data, w, c_init, c_bounds,
                p0_lower=0.0, cfl=0.3, mem=20, iters=20, rtol=1e-4, alpha0=0.1,
                sigma_p0=0.25, c_bg=1500.0, min_pml=20, callback=None, prior=None):
    """Joint reconstruction of p0[K] and c over the multigrid levels.

    ``levels``: domain sides N_l (coarse to fine); ``L``: domain side (m);
    ``y_meas``: data [K][Nt][M] at times n * dt_data; ``w``: weights [K];
    ``c_bounds``: (L_c, U_c), also the reference speed c_ref = U_c.
    ``prior``: None (data term only) or a dict with tau (m), eta_c, sigma_c,
    eta_p0, sigma_p0: the Ornstein-Uhlenbeck prior terms of Eq.
    (Minimised_functional) on each level's grid (oracle/prior.py).
    Returns (p0[K][N][N], c[N][N], history) on the finest level.
    """
    Lc, Uc = c_bounds
    K = y_meas.shape[0]
    p0 = None
    c = None
    hist = []
    for li, nl in enumerate(levels):
        dx = L / nl
        g = make_grid(nl, dx, 1, c_ref=Uc, cfl=cfl, min_pml=min_pml, c_bg=c_bg)
        g.nt = level_nt(T, g.dt)
        S = sensor_matrix(g, sensors_xy)
        yl = time_interp(y_meas, dt_data, g.dt, g.nt)
        if p0 is None:
            p0 = np.zeros((K, nl, nl))
            c = np.full((nl, nl), float(c_init))
        else:
            p0 = prolong(p0, nl)
            c = prolong(c, nl)
        npx = nl * nl
        x0 = np.concatenate([p0.ravel(), c.ravel()])
        lower = np.concatenate([np.full(K * npx, p0_lower), np.full(npx, Lc)])
        upper = np.concatenate([np.full(K * npx, np.inf), np.full(npx, Uc)])
        scale = np.concatenate([np.full(K * npx, sigma_p0), np.full(npx, (Uc - Lc) / 4.0)])

        pr = OUPrior((nl, nl), dx, prior["tau"]) if prior else None

        def unpack(x):
            return x[:K * npx].reshape(K, nl, nl), x[K * npx:].reshape(nl, nl)

        def prior_part(pp, cc):
            return prior_value_grad(pr, pp, cc, prior["eta_p0"], prior["sigma_p0"], prior["eta_c"],
                                    prior["sigma_c"])

        def fun(x):
            pp, cc = unpack(x)
            J = objective(g, cc, pp, S, yl, w)[0]
            return J + (prior_part(pp, cc)[0] if pr else 0.0)

        def fun_grad(x):
            pp, cc = unpack(x)
            J, gp, gc = adjoint_grad(g, cc, pp, S, yl, w)
            if pr:
                Jp, gpp, gcp = prior_part(pp, cc)
                J, gp, gc = J + Jp, gp + gpp, gc + gcp
            return J, np.concatenate([gp.ravel(), gc.ravel()])

        res = projected_lbfgs(fun, fun_grad, x0, lower, upper, scale, mem=mem, max_iter=iters,
                              alpha0=alpha0, rtol=rtol,
                              callback=(lambda it, x, J: callback(li, it, x, J)) if callback else None)
        p0, c = unpack(res.x)
        hist.append(dict(level=li, n=nl, nt=g.nt, pml=g.pml, result=res))
    return p0, c, hist
