"""Forward solve f^i : (p0^i, c) -> y^i and the discrete energy (oracle, FP64).

Implements the k-space pseudospectral time stepping that approximates the
acoustic initial value problem (Eq. WaveEquation, Sec. 2.1) and the
observation model y = f(x) + e (Eq. ObservationModel, Sec. 2.2):

  initial condition (p(t=0) = p0, dp/dt(t=0) = 0):
      p^0 = p0,  rho_x^0 = rho_y^0 = p0 / (2 c^2),
      u^{-1/2} = + dt/(2 rho0) G p0          (makes p^{-1} = p^{+1})
  for n = 0 .. Nt-2:
      u^{n+1/2}   = a' (a' u^{n-1/2} - dt/rho0 G p^n)           (per axis)
      rho^{n+1}   = a  (a  rho^n     - dt rho0 D u^{n+1/2})     (per axis)
      p^{n+1}     = c^2 (rho_x^{n+1} + rho_y^{n+1})
  samples y^n = S p^n for n = 0 .. Nt-1 (t_n = n dt).

The K data sets share c and are independent otherwise.
"""
from __future__ import annotations

import numpy as np


def initial_state(grid, c_full, p0):
    """State (ux, uy, rx, ry, p) at n = 0 for p0 on the grid ([..][ng][ng])."""
    dt, rho0 = grid.dt, grid.rho0
    c2 = c_full ** 2
    rx = p0 / (2.0 * c2)
    ry = p0 / (2.0 * c2)
    ux = (dt / (2.0 * rho0)) * grid.Gx(p0)
    uy = (dt / (2.0 * rho0)) * grid.Gy(p0)
    return ux, uy, rx, ry, p0.copy()


def step(grid, c_full, ux, uy, rx, ry, p):
    """One time step n -> n+1 of the split-field k-space scheme."""
    dt, rho0 = grid.dt, grid.rho0
    ux = grid.asx * (grid.asx * ux - (dt / rho0) * grid.Gx(p))
    uy = grid.asy * (grid.asy * uy - (dt / rho0) * grid.Gy(p))
    rx = grid.ax * (grid.ax * rx - dt * rho0 * grid.Dx(ux))
    ry = grid.ay * (grid.ay * ry - dt * rho0 * grid.Dy(uy))
    p = c_full ** 2 * (rx + ry)
    return ux, uy, rx, ry, p


def forward(grid, c_dom, p0_dom, S, keep_history: bool = False):
    """Sensor traces y[K][Nt][M] for initial pressures p0_dom[K][n][n].

    With ``keep_history`` also returns rho_x + rho_y on the grid for every n
    (``[K][Nt][ng][ng]``), which the adjoint needs.
    """
    p0_dom = np.asarray(p0_dom, dtype=np.float64)
    if p0_dom.ndim == 2:
        p0_dom = p0_dom[None]
    K = p0_dom.shape[0]
    c_full = grid.medium(c_dom)
    p0 = grid.pad(p0_dom)
    M = S.shape[0]
    y = np.zeros((K, grid.nt, M))
    hist = np.zeros((K, grid.nt, grid.ng, grid.ng)) if keep_history else None
    ux, uy, rx, ry, p = initial_state(grid, c_full, p0)
    for n in range(grid.nt):
        if n > 0:
            ux, uy, rx, ry, p = step(grid, c_full, ux, uy, rx, ry, p)
        for k in range(K):
            y[k, n] = S @ p[k].ravel()
        if keep_history:
            hist[:, n] = rx + ry
    return (y, hist) if keep_history else y


def pressure_fields(grid, c_full, p0, nsteps: int):
    """p^n on the grid for n = 0..nsteps (list), starting from grid field p0."""
    ux, uy, rx, ry, p = initial_state(grid, c_full, p0)
    out = [p.copy()]
    for _ in range(nsteps):
        ux, uy, rx, ry, p = step(grid, c_full, ux, uy, rx, ry, p)
        out.append(p.copy())
    return out


def energy_history(grid, c_full, p0, nsteps: int):
    """Discrete acoustic energy E^n for n = 0..nsteps-1.

    E^n = rho0/2 sum u^{n-1/2} . u^{n+1/2} + sum (p^n)^2 / (2 rho0 c^2).
    Without the PML this is conserved exactly by the staggered leapfrog
    because G^T = -D; with the PML it decays.
    """
    rho0 = grid.rho0
    c2 = c_full ** 2
    ux, uy, rx, ry, p = initial_state(grid, c_full, p0)
    E = []
    for _ in range(nsteps):
        ux1, uy1, rx1, ry1, p1 = step(grid, c_full, ux, uy, rx, ry, p)
        e = 0.5 * rho0 * np.sum(ux * ux1 + uy * uy1) + np.sum(p * p / (2.0 * rho0 * c2))
        E.append(e)
        ux, uy, rx, ry, p = ux1, uy1, rx1, ry1, p1
    return np.array(E)
