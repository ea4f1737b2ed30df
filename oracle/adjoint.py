"""Objective and exact discrete adjoint gradient (oracle, FP64).

Objective, data term of Eq. (Minimised_functional):
    J = sum_k 1/2 || L_e^k (y_k - f_k(x)) ||^2 = sum_k w_k/2 || S p_k - y_k ||^2
with L_e^T L_e = w_k I (noise std = 1 % of each data set's peak-to-peak value, Sec. 4.1.2).

The paper computes the gradient with the adjoint-state method: the adjoint
wave equation driven by the time-reversed weighted residual (Eq.
AdjointEquation), dJ/dp0 = q(T) (Eq. gradient_p0) and dJ/dc = sum_k int
(-2/c^3 p_tt) q(T-t) dt (Eq. gradient_sos).  Here the same quantities are
computed for the DISCRETE forward of ``oracle.forward``: reverse mode of each
step, with the residual r^n = w_k (S p^n - y^n) injected at the sensors in
reverse time (the sign makes dJ/dp0 = +q(T)).  Starting from zero adjoint
states, for n = Nt-1 .. 1:
    pb^n       += S^T r^n
    rb_{x,y}^n += c^2 pb^n ;  cb += 2 c (rho_x^n + rho_y^n) pb^n
    t           = a rb^n ;  rb^{n-1} = a t ;  ub^{n-1/2} += dt rho0 G t
    t'          = a' ub^{n-1/2} ;  ub^{n-3/2} = a' t' ;  pb^{n-1} = dt/rho0 D.t'
and at n = 0 (transposes of the initial condition):
    pb^0 += S^T r^0
    dJ/dp0 = pb^0 + (rb_x^0 + rb_y^0)/(2 c^2) - dt/(2 rho0) D.ub^{-1/2}
    cb    += -(rb_x^0 + rb_y^0) p0 / c^3
The transposes use G^T = -D.  The gradient is restricted to the domain; c in
the PML is fixed (c_bg) and not an unknown.
"""
from __future__ import annotations

import numpy as np

from .forward import forward


def objective(grid, c_dom, p0_dom, S, y_meas, w):
    """J (float) and predicted traces."""
    y = forward(grid, c_dom, p0_dom, S)
    d = y - y_meas
    J = 0.5 * float(np.sum(np.asarray(w)[:, None, None] * d * d))
    return J, y


def _reverse(grid, c_full, p0, S, r, rsum_hist=None):
    """Reverse sweep; returns (dJ/dp0 on the grid [K][ng][ng], cb [K][ng][ng]).

    ``r`` is the weighted residual [K][Nt][M]; with ``rsum_hist`` None the
    c-terms are skipped (linear adjoint A^T : r -> dJ/dp0 at fixed c).
    """
    dt, rho0 = grid.dt, grid.rho0
    K, nt, _ = r.shape
    ng = grid.ng
    c2 = c_full ** 2
    ST = S.T.tocsr()
    pb = np.zeros((K, ng, ng))
    rbx = np.zeros((K, ng, ng))
    rby = np.zeros((K, ng, ng))
    ubx = np.zeros((K, ng, ng))
    uby = np.zeros((K, ng, ng))
    cb = np.zeros((K, ng, ng))
    for n in range(nt - 1, 0, -1):
        for k in range(K):
            pb[k] += (ST @ r[k, n]).reshape(ng, ng)
        rbx = rbx + c2 * pb
        rby = rby + c2 * pb
        if rsum_hist is not None:
            cb += 2.0 * c_full * rsum_hist[:, n] * pb
        tx = grid.ax * rbx
        ty = grid.ay * rby
        rbx = grid.ax * tx
        rby = grid.ay * ty
        ubx = ubx + dt * rho0 * grid.Gx(tx)
        uby = uby + dt * rho0 * grid.Gy(ty)
        tpx = grid.asx * ubx
        tpy = grid.asy * uby
        ubx = grid.asx * tpx
        uby = grid.asy * tpy
        pb = (dt / rho0) * (grid.Dx(tpx) + grid.Dy(tpy))
    for k in range(K):
        pb[k] += (ST @ r[k, 0]).reshape(ng, ng)
    p0b = pb + (rbx + rby) / (2.0 * c2) - (dt / (2.0 * rho0)) * (grid.Dx(ubx) + grid.Dy(uby))
    if rsum_hist is not None:
        cb += -(rbx + rby) * p0 / (c_full ** 3)
    return p0b, cb


def adjoint_grad(grid, c_dom, p0_dom, S, y_meas, w):
    """J, dJ/dp0 [K][n][n], dJ/dc [n][n] for the data term of Eq. (Minimised_functional)."""
    p0_dom = np.asarray(p0_dom, dtype=np.float64)
    if p0_dom.ndim == 2:
        p0_dom = p0_dom[None]
    w = np.asarray(w, dtype=np.float64)
    y, hist = forward(grid, c_dom, p0_dom, S, keep_history=True)
    d = y - np.asarray(y_meas, dtype=np.float64)
    J = 0.5 * float(np.sum(w[:, None, None] * d * d))
    r = w[:, None, None] * d
    c_full = grid.medium(c_dom)
    p0b, cb = _reverse(grid, c_full, grid.pad(p0_dom), S, r, rsum_hist=hist)
    return J, grid.crop(p0b), grid.crop(cb.sum(axis=0))


def adjoint_linear(grid, c_dom, S, r):
    """A^T r for the linear map A_c : p0 -> y at fixed c (returns [K][n][n])."""
    r = np.asarray(r, dtype=np.float64)
    K = r.shape[0]
    c_full = grid.medium(c_dom)
    p0b, _ = _reverse(grid, c_full, np.zeros((K, grid.ng, grid.ng)), S, r, rsum_hist=None)
    return grid.crop(p0b)
