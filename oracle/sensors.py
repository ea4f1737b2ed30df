"""Point-sensor sampling matrix S (oracle, FP64).

Sec. 4 uses point-like acoustic sensors; on the coarse multigrid levels the
sensors fall between grid points (Table 1, sensor layer N_z^S), so each sample
is the bilinear interpolation of the pressure at the sensor's physical
position.  Grid cell (gy, gx) has its centre at ((gx - P + 0.5) dx,
(gy - P + 0.5) dx) in the domain frame (origin at the domain's lower-left
corner).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def sensor_matrix(grid, xy: np.ndarray) -> sp.csr_matrix:
    """Sparse S with shape (M, ng*ng): y_m = sum_j S[m, j] p.ravel()[j].

    ``xy`` is ``[M][2]`` (x, y) in metres.  Raises ValueError if a sensor's
    2 x 2 stencil leaves the grid.
    """
    xy = np.asarray(xy, dtype=np.float64)
    ng, P, dx = grid.ng, grid.pml, grid.dx
    rows, cols, vals = [], [], []
    for m, (sx, sy) in enumerate(xy):
        gx = sx / dx - 0.5 + P
        gy = sy / dx - 0.5 + P
        ix, iy = int(np.floor(gx)), int(np.floor(gy))
        fx, fy = gx - ix, gy - iy
        if ix < 0 or iy < 0 or ix + 1 > ng - 1 or iy + 1 > ng - 1:
            raise ValueError(f"sensor {m} at ({sx}, {sy}) m lies outside the grid")
        for dy_, wy in ((0, 1.0 - fy), (1, fy)):
            for dx_, wx in ((0, 1.0 - fx), (1, fx)):
                rows.append(m)
                cols.append((iy + dy_) * ng + (ix + dx_))
                vals.append(wx * wy)
    return sp.csr_matrix((vals, (rows, cols)), shape=(xy.shape[0], ng * ng))
