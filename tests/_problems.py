"""Shared problem builders for the parity tests (inputs from pat_synth only)."""
from __future__ import annotations

import numpy as np

import pat_synth as ps


def grid_params(n, nt, dx=1e-4, c_hi=1750.0, cfl=0.3, min_pml=20, pml=None, pml_alpha=2.0, c_bg=1500.0):
    from oracle.grid import pml_auto
    P = pml_auto(n, min_pml) if pml is None else pml
    return dict(n=n, pml=P, dx=dx, dt=cfl * dx / c_hi, nt=nt, c_ref=c_hi, rho0=1000.0, pml_alpha=pml_alpha,
                c_bg=c_bg)


def oracle_grid(gp):
    from oracle.grid import Grid
    return Grid(n=gp["n"], pml=gp["pml"], dx=gp["dx"], dt=gp["dt"], nt=gp["nt"], c_ref=gp["c_ref"],
                rho0=gp["rho0"], alpha_max=gp["pml_alpha"], c_bg=gp["c_bg"])


def gpu_plan(gp, sensors, K, ckpt_every=32):
    from paper_2505_08482_gb300.solver import GridSpec, Plan
    return Plan(GridSpec(**gp), sensors, K, ckpt_every=ckpt_every)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def small_case(n=40, K=3, M=20, nt=150, seed=5):
    """Ragged small case: several tiles per pass with partial last tiles."""
    rng = ps.rng_for(seed)
    c = ps.ellipse_phantom(n, 3, rng)
    p0 = np.stack([ps.blob_p0(n, 3, rng, sigma_cells=(1.5, 3.0)) for _ in range(K)])
    xy = ps.circle_sensors(n, M, 1e-4, phase=0.3)
    return c, p0, xy
