"""Discrete grid and k-space operators of the forward model (oracle, FP64).

The paper approximates the wave equation (Eq. WaveEquation, Sec. 2.1) with a
k-space pseudospectral method and a PML (Sec. 2.1; Sec. 4.1.1: PML outside the
target and sensor layers, total grid size chosen with small prime factors).
It does not restate the discretisation; the reading used here is the
first-order, split-field, staggered k-space scheme of the cited k-space method:

* wavenumbers k = 2 pi / (Ng dx) * {-floor(Ng/2) .. ceil(Ng/2)-1} in FFT order;
* k-space correction kappa = sinc(c_ref |k| dt / 2), sinc(x) = sin(x)/x;
* gradient operator   G_x = F^-1 diag(i k_x kappa e^{+i k_x dx/2}) F,
  divergence operator D_x = F^-1 diag(i k_x kappa e^{-i k_x dx/2}) F
  (the same along y), so that G_x^T = -D_x exactly;
* PML absorption alpha(xi) = alpha_max (c_ref/dx) (xi/P)^4 at depth xi (cells)
  into the layer, a = exp(-alpha dt / 2), evaluated at cell centres (for the
  density fields) and at +1/2 cell (for the staggered velocities);
* c_ref is fixed per grid (the upper bound of c), so dt, kappa and the PML do
  not depend on the unknown.

Fields are arrays ``[y][x]`` on the Ng x Ng FFT grid; the N x N domain
occupies rows/columns P .. P+N-1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def is_smooth(n: int, primes=(2, 3, 5)) -> bool:
    """True if n factors into the given primes only (Sec. 4.1.1: small prime factors)."""
    if n < 1:
        return False
    for p in primes:
        while n % p == 0:
            n //= p
    return n == 1


def pml_auto(n: int, min_pml: int = 20) -> int:
    """Smallest PML width P >= min_pml with N + 2P even and 5-smooth (Sec. 4.1.1).

    An odd N has no even grid side; that raises ValueError.
    """
    if n % 2:
        raise ValueError("an odd domain side has no even FFT grid side")
    p = min_pml
    while not ((n + 2 * p) % 2 == 0 and is_smooth(n + 2 * p)):
        p += 1
    return p


def time_step(dx: float, cfl: float, c_ref: float) -> float:
    """dt = CFL dx / c_ref (Table 1 uses CFL 0.3 at the reference speed)."""
    return cfl * dx / c_ref


@dataclass
class Grid:
    """Discretisation of one reconstruction level (oracle).

    n: domain side in cells; pml: PML width P; dx: cell size (m); dt: time
    step (s); nt: number of time samples (t_n = n dt, n = 0..nt-1); c_ref:
    reference speed in kappa and the PML; rho0: uniform density; alpha_max:
    PML strength in nepers per cell at the outer edge; c_bg: speed of sound
    outside the domain.
    """
    n: int
    pml: int
    dx: float
    dt: float
    nt: int
    c_ref: float
    rho0: float = 1000.0
    alpha_max: float = 2.0
    c_bg: float = 1500.0
    ng: int = field(init=False)

    def __post_init__(self):
        self.ng = self.n + 2 * self.pml
        ng, dx, dt = self.ng, self.dx, self.dt
        # wavenumbers in FFT order: fftfreq gives {0..ceil-1, -floor..-1} / (ng dx)
        k1 = 2.0 * np.pi * np.fft.fftfreq(ng, d=dx)
        self.k1 = k1
        self.KX = np.broadcast_to(k1[None, :], (ng, ng)).copy()
        self.KY = np.broadcast_to(k1[:, None], (ng, ng)).copy()
        kabs = np.sqrt(self.KX ** 2 + self.KY ** 2)
        arg = 0.5 * self.c_ref * kabs * dt
        with np.errstate(invalid="ignore", divide="ignore"):
            self.kappa = np.where(arg == 0.0, 1.0, np.sin(arg) / np.where(arg == 0.0, 1.0, arg))
        self.mGx = 1j * self.KX * self.kappa * np.exp(+0.5j * self.KX * dx)
        self.mGy = 1j * self.KY * self.kappa * np.exp(+0.5j * self.KY * dx)
        self.mDx = 1j * self.KX * self.kappa * np.exp(-0.5j * self.KX * dx)
        self.mDy = 1j * self.KY * self.kappa * np.exp(-0.5j * self.KY * dx)
        g = np.arange(ng, dtype=np.float64)
        self.a_cell = self.pml_factor(g)          # at cell centres
        self.a_stag = self.pml_factor(g + 0.5)    # at +1/2 cell
        # 2-D broadcasts: x-profiles vary along columns, y-profiles along rows
        self.ax = self.a_cell[None, :]
        self.ay = self.a_cell[:, None]
        self.asx = self.a_stag[None, :]
        self.asy = self.a_stag[:, None]

    def depth(self, s: np.ndarray) -> np.ndarray:
        """Depth (cells) of position s into the PML; 0 inside the domain's cell centres."""
        lo = self.pml - s
        hi = s - (self.pml + self.n - 1)
        return np.maximum(0.0, np.maximum(lo, hi))

    def pml_factor(self, s: np.ndarray) -> np.ndarray:
        """a(s) = exp(-alpha(s) dt / 2), alpha = alpha_max (c_ref/dx) (xi/P)^4."""
        if self.pml == 0 or self.alpha_max == 0.0:
            return np.ones_like(s, dtype=np.float64)
        xi = self.depth(s)
        alpha = self.alpha_max * (self.c_ref / self.dx) * (xi / self.pml) ** 4
        return np.exp(-0.5 * alpha * self.dt)

    # ---- operators (plain full complex 2-D FFTs) ----
    @staticmethod
    def apply(mult: np.ndarray, f: np.ndarray) -> np.ndarray:
        """F^-1 diag(mult) F f over the last two axes; real part (mult is Hermitian)."""
        return np.real(np.fft.ifft2(mult * np.fft.fft2(f, axes=(-2, -1)), axes=(-2, -1)))

    def Gx(self, f):
        return self.apply(self.mGx, f)

    def Gy(self, f):
        return self.apply(self.mGy, f)

    def Dx(self, f):
        return self.apply(self.mDx, f)

    def Dy(self, f):
        return self.apply(self.mDy, f)

    # ---- medium and padding (Sec. 2.1; PML lies outside the domain) ----
    def pad(self, f_dom: np.ndarray) -> np.ndarray:
        """Zero-pad domain fields [..][n][n] into the FFT grid [..][ng][ng]."""
        f_dom = np.asarray(f_dom, dtype=np.float64)
        out = np.zeros(f_dom.shape[:-2] + (self.ng, self.ng))
        P, n = self.pml, self.n
        out[..., P:P + n, P:P + n] = f_dom
        return out

    def crop(self, f: np.ndarray) -> np.ndarray:
        """Domain part [..][n][n] of a grid field."""
        P, n = self.pml, self.n
        return f[..., P:P + n, P:P + n]

    def medium(self, c_dom: np.ndarray) -> np.ndarray:
        """Speed of sound on the whole grid: c on the domain, c_bg elsewhere."""
        c = np.full((self.ng, self.ng), float(self.c_bg))
        P, n = self.pml, self.n
        c[P:P + n, P:P + n] = np.asarray(c_dom, dtype=np.float64)
        return c


def make_grid(n: int, dx: float, nt: int, c_ref: float, cfl: float = 0.3, pml: int | None = None,
              min_pml: int = 20, **kw) -> Grid:
    """Grid with dt from the CFL rule and an automatic 5-smooth PML width."""
    if pml is None:
        pml = pml_auto(n, min_pml)
    return Grid(n=n, pml=pml, dx=dx, dt=time_step(dx, cfl, c_ref), nt=nt, c_ref=c_ref, **kw)
