"""Seeded phantom, sensor and noise generators (inputs only).

All generators take a ``numpy.random.Generator`` built on PCG64 so that the
same seed gives the same arrays on every machine.  Arrays are float64; the GPU
side converts them to float32 when it uploads them.

Index convention: a field on the N x N domain is ``[y][x]`` with x fastest;
cell (iy, ix) has its centre at ((ix + 0.5) dx, (iy + 0.5) dx) in the domain
frame, whose origin is the domain's lower-left corner.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng_for(seed: int) -> np.random.Generator:
    """PCG64 generator for ``seed``."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def _cell_coords(n: int):
    """Cell-centre coordinates in cells, origin at the domain centre."""
    t = np.arange(n, dtype=np.float64) + 0.5 - n / 2.0
    yy, xx = np.meshgrid(t, t, indexing="ij")
    return xx, yy


def ellipse_phantom(n: int, n_incl: int, rng: np.random.Generator,
                    c_bg: float = 1500.0, c_range=(1400.0, 1650.0)) -> np.ndarray:
    """Speed of sound: background ``c_bg`` plus ``n_incl`` elliptical inclusions.

    Centres are uniform in a disc of radius 0.3 n, semi-axes uniform in
    [0.05 n, 0.15 n], orientation uniform in [0, pi), value uniform in
    ``c_range``; a later ellipse overwrites an earlier one where they overlap.
    """
    xx, yy = _cell_coords(n)
    c = np.full((n, n), float(c_bg))
    for _ in range(n_incl):
        r = 0.3 * n * np.sqrt(rng.uniform())
        phi = rng.uniform(0.0, 2.0 * np.pi)
        cx, cy = r * np.cos(phi), r * np.sin(phi)
        a = rng.uniform(0.05 * n, 0.15 * n)
        b = rng.uniform(0.05 * n, 0.15 * n)
        th = rng.uniform(0.0, np.pi)
        val = rng.uniform(*c_range)
        dx, dy = xx - cx, yy - cy
        u = dx * np.cos(th) + dy * np.sin(th)
        v = -dx * np.sin(th) + dy * np.cos(th)
        c[(u / a) ** 2 + (v / b) ** 2 <= 1.0] = val
    return c


def blob_p0(n: int, n_blobs: int, rng: np.random.Generator,
            amp=(0.5, 1.0), sigma_cells=(2.0, 5.0), radius_frac: float = 0.35) -> np.ndarray:
    """Initial pressure made of ``n_blobs`` Gaussian blobs (summed).

    Centres uniform in a disc of radius ``radius_frac`` n, amplitude and width
    (in cells) uniform in the given ranges.
    """
    xx, yy = _cell_coords(n)
    p0 = np.zeros((n, n))
    for _ in range(n_blobs):
        r = radius_frac * n * np.sqrt(rng.uniform())
        phi = rng.uniform(0.0, 2.0 * np.pi)
        cx, cy = r * np.cos(phi), r * np.sin(phi)
        a = rng.uniform(*amp)
        s = rng.uniform(*sigma_cells)
        p0 += a * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2.0 * s * s))
    return p0


def vessel_p0(n: int, rng: np.random.Generator, n_seg=(3, 6), sigma_cells=(1.0, 2.5),
              length_frac=(0.1, 0.4), amp=(0.5, 1.0), radius_frac: float = 0.35) -> np.ndarray:
    """Vessel-like initial pressure: Gaussian line segments, summed, clipped at 1.

    Each segment has a Gaussian cross-section of width U(sigma_cells) cells,
    length U(length_frac) n, amplitude U(amp); its centre lies in a disc of
    radius ``radius_frac`` n.
    """
    xx, yy = _cell_coords(n)
    p0 = np.zeros((n, n))
    for _ in range(int(rng.integers(n_seg[0], n_seg[1] + 1))):
        r = radius_frac * n * np.sqrt(rng.uniform())
        phi = rng.uniform(0.0, 2.0 * np.pi)
        cx, cy = r * np.cos(phi), r * np.sin(phi)
        th = rng.uniform(0.0, np.pi)
        half = 0.5 * rng.uniform(*length_frac) * n
        s = rng.uniform(*sigma_cells)
        a = rng.uniform(*amp)
        ex, ey = np.cos(th), np.sin(th)
        dx, dy = xx - cx, yy - cy
        along = np.clip(dx * ex + dy * ey, -half, half)
        px, py = cx + along * ex, cy + along * ey
        d2 = (xx - px) ** 2 + (yy - py) ** 2
        p0 += a * np.exp(-d2 / (2.0 * s * s))
    return np.minimum(p0, 1.0)


def circle_sensors(n: int, m: int, dx: float, radius_cells: float | None = None,
                   phase: float = 0.0) -> np.ndarray:
    """``m`` point sensors evenly spaced on a circle about the domain centre.

    Returns ``[m][2]`` (x, y) positions in metres in the domain frame (origin at
    the lower-left corner of the N x N domain).  The default radius is
    0.4375 n cells (28 cells at n = 64).
    """
    if radius_cells is None:
        radius_cells = 0.4375 * n
    ang = phase + 2.0 * np.pi * np.arange(m) / m
    ctr = 0.5 * n * dx
    xy = np.empty((m, 2))
    xy[:, 0] = ctr + radius_cells * dx * np.cos(ang)
    xy[:, 1] = ctr + radius_cells * dx * np.sin(ang)
    return xy


def add_noise(y_clean: np.ndarray, rng: np.random.Generator, rel: float = 0.01) -> np.ndarray:
    """Additive Gaussian noise, std = ``rel`` x peak-to-peak of each data set.

    ``y_clean`` is ``[K][Nt][M]``; data set k gets its own standard deviation
    (Sec. 4.1.1: standard deviation 1 % of the clean data set's peak-to-peak value).
    """
    y = np.asarray(y_clean, dtype=np.float64)
    out = np.empty_like(y)
    for k in range(y.shape[0]):
        sig = rel * (y[k].max() - y[k].min())
        out[k] = y[k] + sig * rng.standard_normal(y[k].shape)
    return out


def noise_weights(y_noisy: np.ndarray, rel: float = 0.01) -> np.ndarray:
    """Per-data-set weights w_k = 1 / sigma_k^2 with sigma_k = rel x p2p(noisy y_k).

    For the reconstruction the noise level is taken from the noisy data's
    peak-to-peak value (Sec. 4.1.2); L_e^T L_e = w_k I.
    """
    y = np.asarray(y_noisy, dtype=np.float64)
    w = np.empty(y.shape[0])
    for k in range(y.shape[0]):
        sig = rel * (y[k].max() - y[k].min())
        w[k] = 1.0 / (sig * sig) if sig > 0 else 1.0
    return w


@dataclass
class Workload:
    """One synthetic reconstruction problem (domain fields, float64)."""
    n: int
    dx: float
    nt: int
    c_true: np.ndarray            # [n][n]
    p0_true: np.ndarray           # [K][n][n]
    sensors: np.ndarray           # [M][2] metres
    c_bg: float = 1500.0
    c_bounds: tuple = (1350.0, 1750.0)
    cfl: float = 0.3
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def k(self) -> int:
        return self.p0_true.shape[0]

    @property
    def m(self) -> int:
        return self.sensors.shape[0]


def workload(name: str, seed: int = 0) -> Workload:
    """Named synthetic workloads.

    * ``"plain64"``: 64 x 64, dx 0.1 mm, 3 ellipses, K = 1 with 5 blobs,
      64 sensors on a circle of radius 28 cells, Nt = 400.
    * ``"vessels128"``: 128 x 128, 6 ellipses, K = 4 vessel sets, 256 sensors,
      Nt = 900 (dx 0.1 mm).
    * ``"vessels256"``: 256 x 256, 6 ellipses, K = 8 vessel sets, 512 sensors,
      Nt = 1800 (dx 0.1 mm).
    * ``"tiny16"``: 16 x 16, K = 2, 12 sensors, Nt = 60 (finite-difference size).
    """
    rng = rng_for(seed)
    dx = 1e-4
    if name == "plain64":
        n, K, M, nt = 64, 1, 64, 400
        c = ellipse_phantom(n, 3, rng)
        p0 = np.stack([blob_p0(n, 5, rng) for _ in range(K)])
    elif name == "vessels128":
        n, K, M, nt = 128, 4, 256, 900
        c = ellipse_phantom(n, 6, rng)
        p0 = np.stack([vessel_p0(n, rng) for _ in range(K)])
    elif name == "vessels256":
        n, K, M, nt = 256, 8, 512, 1800
        c = ellipse_phantom(n, 6, rng)
        p0 = np.stack([vessel_p0(n, rng) for _ in range(K)])
    elif name == "tiny16":
        n, K, M, nt = 16, 2, 12, 60
        c = ellipse_phantom(n, 2, rng)
        p0 = np.stack([blob_p0(n, 2, rng, sigma_cells=(1.5, 2.5)) for _ in range(K)])
    else:
        raise ValueError(f"unknown workload {name!r}")
    sensors = circle_sensors(n, M, dx)
    return Workload(n=n, dx=dx, nt=nt, c_true=c, p0_true=p0, sensors=sensors, seed=seed)


def add_noise_torch(y, gen, rel: float = 0.01):
    """Torch (GPU) version of add_noise for large training sets: y [K][Nt][M] per data set.

    Returns (noisy y, weights 1/(rel p2p(noisy))^2) with a seeded torch.Generator on y's device.
    """
    import torch
    p2p = (y.amax(dim=(1, 2)) - y.amin(dim=(1, 2))).clamp_min(1e-30)
    noise = torch.randn(y.shape, generator=gen, device=y.device, dtype=y.dtype)
    yn = y + (rel * p2p)[:, None, None] * noise
    p2pn = (yn.amax(dim=(1, 2)) - yn.amin(dim=(1, 2))).clamp_min(1e-30)
    return yn, 1.0 / (rel * p2pn) ** 2


def warmstart_sample(n: int, K: int, seed: int):
    """c with 2-8 random inclusions in [1400, 1650] m/s and K vessel-like p0 sets (learned warm start data)."""
    rng = rng_for(seed)
    c = ellipse_phantom(n, int(rng.integers(2, 9)), rng)
    p0 = np.stack([vessel_p0(n, rng) for _ in range(K)])
    return c, p0


# ---------------------------------------------------------------------------
# Simple-phantom geometry of Sec. 4.1.1 (stand-in: the paper shows the shapes only in
# figures).  A 20 mm x 20 mm target sits in a computational domain with a sensor layer of
# `margin` metres on every side; 236 point sensors lie evenly on the square 0.2 mm outside
# the target boundary.

SIMPLE_TARGET = 20e-3      # target side (m)
SIMPLE_MARGIN = 0.64e-3    # sensor layer on each side (10 data-grid pixels of 63.7 um)
SIMPLE_L = SIMPLE_TARGET + 2 * SIMPLE_MARGIN


def square_sensors(m: int = 236, offset: float = 0.2e-3, target: float = SIMPLE_TARGET,
                   margin: float = SIMPLE_MARGIN) -> np.ndarray:
    """``m`` sensors evenly spaced (by arc length) on the square ``offset`` outside the target.

    Returns ``[m][2]`` (x, y) in metres in the domain frame.
    """
    side = target + 2.0 * offset
    lo = margin - offset
    s = (np.arange(m) + 0.5) * (4.0 * side / m)
    xy = np.empty((m, 2))
    for i, t in enumerate(s):
        e, u = int(t // side), t % side
        xy[i] = [(lo + u, lo), (lo + side, lo + u), (lo + side - u, lo + side), (lo, lo + side - u)][e]
    return xy


def _disc(n: int, L: float, cx: float, cy: float, r: float) -> np.ndarray:
    """Area fraction of each cell inside the disc (4 x 4 sub-samples per cell)."""
    dx = L / n
    sub = (np.arange(4) + 0.5) / 4.0
    acc = np.zeros((n, n))
    for sy in sub:
        for sx in sub:
            x = (np.arange(n) + sx) * dx
            y = (np.arange(n) + sy) * dx
            acc += ((x[None, :] - cx) ** 2 + (y[:, None] - cy) ** 2) <= r * r
    return acc / 16.0


def _rect(n: int, L: float, x0: float, x1: float, y0: float, y1: float) -> np.ndarray:
    dx = L / n
    sub = (np.arange(4) + 0.5) / 4.0
    acc = np.zeros((n, n))
    for sy in sub:
        for sx in sub:
            x = (np.arange(n) + sx) * dx
            y = (np.arange(n) + sy) * dx
            acc += ((x[None, :] >= x0) & (x[None, :] < x1)) & ((y[:, None] >= y0) & (y[:, None] < y1))
    return acc / 16.0


def simple_phantom_c(kind: str, n: int, L: float = SIMPLE_L, margin: float = SIMPLE_MARGIN) -> np.ndarray:
    """Speed of sound of the simple phantoms on an n x n grid over the domain of side L.

    kind "circles": nine circular inclusions (1580 m/s, radius 1.6 mm, 3 x 3 lattice with
    6 mm pitch) in a 1430 m/s background; "water": the same plus a 3 mm water layer
    (1482 m/s) along the lower target edge; "bone": the circles plus a 6 mm x 2 mm
    rectangular inclusion of 2500 m/s.  Cells are area-averaged.
    """
    c0 = SIMPLE_TARGET / 2.0 + margin
    c = np.full((n, n), 1430.0)
    if kind == "water":
        f = _rect(n, L, 0.0, L, 0.0, margin + 3e-3)
        c = c * (1.0 - f) + 1482.0 * f
    for iy in (-1, 0, 1):
        for ix in (-1, 0, 1):
            f = _disc(n, L, c0 + 6e-3 * ix, c0 + 6e-3 * iy, 1.6e-3)
            c = c * (1.0 - f) + 1580.0 * f
    if kind == "bone":
        f = _rect(n, L, c0 - 3e-3, c0 + 3e-3, c0 + 2e-3, c0 + 4e-3)
        c = c * (1.0 - f) + 2500.0 * f
    return c


def simple_phantom_p0(n: int, K: int = 4, seed: int = 0, L: float = SIMPLE_L,
                      margin: float = SIMPLE_MARGIN) -> np.ndarray:
    """K initial pressures of circular inclusions (10 Pa) in a zero background.

    Each p0_k holds 4-6 discs of radius 0.6-1.6 mm at seeded positions inside the target.
    """
    rng = rng_for(7000 + seed)
    out = np.zeros((K, n, n))
    for k in range(K):
        for _ in range(int(rng.integers(4, 7))):
            r = rng.uniform(0.6e-3, 1.6e-3)
            cx, cy = rng.uniform(margin + 2.5e-3, margin + SIMPLE_TARGET - 2.5e-3, size=2)
            out[k] = np.maximum(out[k], 10.0 * _disc(n, L, cx, cy, r))
    return out
