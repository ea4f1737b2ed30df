"""Pins of the time-grid rules against the discretisations printed in Table 1.

* dt = CFL dz / c with CFL 0.3 at c = 1580 m/s (the inclusion speed) reproduces
  every printed time step to within the printed precision (level 2 to 0.1 %).
* Nt_l = round(T / dt_l) + 1 with T = (Nt - 1) dt of the data grid reproduces
  the printed N_t of every multigrid level from its printed dt.
"""
import os

import pytest

from oracle.grid import time_step, is_smooth
from oracle.multigrid import level_nt

HERE = os.path.dirname(os.path.abspath(__file__))


def _rows():
    rows = []
    with open(os.path.join(HERE, "golden", "table1_discretisation.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, dz, nz, ns, npml, dt, nt = line.split()
            rows.append((name, float(dz), int(nz), int(ns), int(npml), float(dt), int(nt)))
    return rows


def test_cfl_rule_reproduces_dt_column():
    for name, dz, nz, ns, npml, dt, nt in _rows():
        got = time_step(dz * 1e-6, 0.3, 1580.0) * 1e9
        assert abs(got - dt) / dt < 2e-3, (name, got, dt)


def test_nt_rule_reproduces_nt_column():
    rows = _rows()
    data = rows[0]
    T = (data[6] - 1) * data[5] * 1e-9
    for name, dz, nz, ns, npml, dt, nt in rows[1:]:
        assert level_nt(T, dt * 1e-9) == nt, name


def test_reconstruction_grids_are_smooth():
    # the paper sizes the PML so that the total grid has small prime factors
    for name, dz, nz, ns, npml, dt, nt in _rows()[1:]:
        assert is_smooth(nz + 2 * ns + 2 * npml, (2, 3, 5, 7)), name


@pytest.mark.parametrize("n,pml", [(64, 22), (96, 24), (128, 26), (160, 20), (192, 24), (256, 22)])
def test_pml_auto_sizes(n, pml):
    from oracle.grid import pml_auto
    assert pml_auto(n) == pml
    assert is_smooth(n + 2 * pml) and (n + 2 * pml) % 2 == 0
