"""Torch-facing wrapper of the C ABI: plans, workspaces, forward and gradient.

Device memory and streams come from PyTorch; every computation runs in the
CUDA kernels of ``libpat.so`` (there is no CPU or PyTorch fallback).
"""
from __future__ import annotations

import ctypes
import dataclasses
import hashlib
import io
import json
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import _binding as B


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _f32(t, shape, name, device):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}, plan is on {device}")
    return t


def pml_auto(n: int, min_pml: int = 20) -> int:
    """Smallest PML width >= min_pml giving a valid FFT grid (library rule)."""
    return int(B.lib().pat_pml_auto(int(n), int(min_pml)))


@dataclass
class GridSpec:
    n: int
    pml: int
    dx: float
    dt: float
    nt: int
    c_ref: float
    rho0: float = 1000.0
    pml_alpha: float = 2.0
    c_bg: float = 1500.0

    @property
    def ng(self):
        return self.n + 2 * self.pml


class Plan:
    """A solver plan on one grid (wraps pat_plan).

    ``K`` is the number of data sets of one reconstruction, or a sequence
    with the number of data sets of each of several independent
    reconstructions (instances) solved as one batch; then ``c`` and its
    gradient are ``[ninst][n][n]`` and J is ``[ninst]``.
    """

    def __init__(self, grid: GridSpec, sensors_xy, K, ckpt_every: int = 32, device=None):
        self.grid = grid
        if np.ndim(K) == 0:
            self.Ks = [int(K)]
            self.batched = False
        else:
            self.Ks = [int(k) for k in K]
            self.batched = True
        self.ninst = len(self.Ks)
        self.K = int(sum(self.Ks))
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        xy = np.ascontiguousarray(np.asarray(sensors_xy, dtype=np.float64))
        if xy.ndim != 2 or xy.shape[1] != 2:
            raise ValueError("sensors_xy must be [M][2]")
        self.m = xy.shape[0]
        self.nt = grid.nt
        self.n = grid.n
        g = B.PatGrid(grid.n, grid.pml, grid.dx, grid.dt, grid.nt, grid.c_ref, grid.rho0, grid.pml_alpha, grid.c_bg)
        h = ctypes.c_void_p()
        ks = (ctypes.c_int * self.ninst)(*self.Ks)
        with torch.cuda.device(self.device):
            B.check(B.lib().pat_plan_create_batched(ctypes.byref(h), ctypes.byref(g), self.m,
                                                    xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self.ninst,
                                                    ks, int(ckpt_every)), "pat_plan_create_batched")
        self._h = h
        self.ckpt_every = int(ckpt_every)
        self._ws = {}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                B.lib().pat_plan_destroy(h)
            except Exception:
                pass
            self._h = None

    @property
    def ng(self):
        return int(B.lib().pat_plan_ng(self._h))

    @property
    def variants(self) -> int:
        """Number of fixed-size kernel variants for this grid side (0: generic only)."""
        return int(B.lib().pat_plan_variants(self._h))

    @property
    def variant(self) -> int:
        return int(B.lib().pat_plan_variant(self._h))

    @variant.setter
    def variant(self, v: int):
        with torch.cuda.device(self.device):
            B.check(B.lib().pat_plan_set_variant(self._h, int(v)), "pat_plan_set_variant")

    def workspace_bytes(self, kind: int = B.PAT_WS_GRADIENT) -> int:
        return int(B.lib().pat_workspace_bytes(self._h, kind))

    def workspace(self, kind: int = B.PAT_WS_GRADIENT):
        """Cached device workspace (torch uint8 tensor, 512-byte aligned)."""
        ws = self._ws.get(kind)
        if ws is None:
            ws = torch.empty(max(self.workspace_bytes(kind), 256), dtype=torch.uint8, device=self.device)
            self._ws[kind] = ws
        return ws

    def _shapes(self):
        n, K = self.n, self.K
        sc = (self.ninst, n, n) if self.batched else (n, n)
        return sc, (K, n, n), (K, self.nt, self.m)

    def forward(self, c, p0, y=None, keep_checkpoints=False, stream=None, ws=None):
        """Sensor traces y [K][nt][m] (pat_forward)."""
        sc, sp, sy = self._shapes()
        _f32(c, sc, "c", self.device)
        _f32(p0, sp, "p0", self.device)
        if y is None:
            y = torch.empty(sy, dtype=torch.float32, device=self.device)
        _f32(y, sy, "y", self.device)
        kind = B.PAT_WS_GRADIENT if keep_checkpoints else B.PAT_WS_FORWARD
        if ws is None:
            ws = self.workspace(kind)
        B.check(B.lib().pat_forward(self._h, _ptr(c), _ptr(p0), _ptr(y), _ptr(ws), self.workspace_bytes(kind),
                                    _stream(stream)), "pat_forward")
        return y

    def adjoint_grad(self, c, p0, y_meas, w, grad_p0=None, grad_c=None, J=None, y_pred=None, stream=None, ws=None):
        """(J [device float64 scalar], dJ/dp0 [K][n][n], dJ/dc [n][n]) (pat_adjoint_grad)."""
        sc, sp, sy = self._shapes()
        _f32(c, sc, "c", self.device)
        _f32(p0, sp, "p0", self.device)
        _f32(y_meas, sy, "y_meas", self.device)
        _f32(w, (self.K,), "w", self.device)
        if grad_p0 is None:
            grad_p0 = torch.empty(sp, dtype=torch.float32, device=self.device)
        if grad_c is None:
            grad_c = torch.empty(sc, dtype=torch.float32, device=self.device)
        if J is None:
            J = torch.empty((self.ninst,) if self.batched else (), dtype=torch.float64, device=self.device)
        if y_pred is not None:
            _f32(y_pred, sy, "y_pred", self.device)
        if ws is None:
            ws = self.workspace(B.PAT_WS_GRADIENT)
        B.check(B.lib().pat_adjoint_grad(self._h, _ptr(c), _ptr(p0), _ptr(y_meas), _ptr(w), _ptr(grad_p0),
                                         _ptr(grad_c), _ptr(J), _ptr(y_pred), _ptr(ws),
                                         self.workspace_bytes(B.PAT_WS_GRADIENT), _stream(stream)),
                "pat_adjoint_grad")
        return J, grad_p0, grad_c

    def vjp(self, c, p0, ybar, stream=None, ws=None):
        """(df/dp0)^T ybar and sum_k (df_k/dc)^T ybar_k (pat_vjp)."""
        sc, sp, sy = self._shapes()
        _f32(c, sc, "c", self.device)
        _f32(p0, sp, "p0", self.device)
        _f32(ybar, sy, "ybar", self.device)
        gp = torch.empty(sp, dtype=torch.float32, device=self.device)
        gc = torch.empty(sc, dtype=torch.float32, device=self.device)
        if ws is None:
            ws = self.workspace(B.PAT_WS_GRADIENT)
        B.check(B.lib().pat_vjp(self._h, _ptr(c), _ptr(p0), _ptr(ybar), _ptr(gp), _ptr(gc), _ptr(ws),
                                self.workspace_bytes(B.PAT_WS_GRADIENT), _stream(stream)), "pat_vjp")
        return gp, gc

    @property
    def persistent(self) -> bool:
        """Forward sweeps as one persistent launch (pat_plan_set_persistent)."""
        return bool(B.lib().pat_plan_persistent(self._h) == 1)

    @persistent.setter
    def persistent(self, enable: bool):
        with torch.cuda.device(self.device):
            B.check(B.lib().pat_plan_set_persistent(self._h, int(bool(enable))), "pat_plan_set_persistent")

    @property
    def cluster(self) -> bool:
        """Forward sweeps and segment recomputes cluster-resident (pat_plan_set_cluster)."""
        return bool(B.lib().pat_plan_cluster(self._h) == 1)

    @cluster.setter
    def cluster(self, enable: bool):
        with torch.cuda.device(self.device):
            B.check(B.lib().pat_plan_set_cluster(self._h, int(bool(enable))), "pat_plan_set_cluster")

    @property
    def cluster_capacity(self) -> int:
        """Clusters (data sets) of the cluster-resident form the GPU runs at once (0: unavailable)."""
        with torch.cuda.device(self.device):
            return int(B.lib().pat_plan_cluster_capacity(self._h))

    def set_graphs(self, enable: bool = True):
        """Capture whole calls into CUDA graphs and replay them (pat_plan_set_graphs)."""
        B.check(B.lib().pat_plan_set_graphs(self._h, int(bool(enable))), "pat_plan_set_graphs")

    def autotune(self, stream=None, gradient=True):
        """Time every kernel variant on this GPU and keep the fastest (pat_plan_autotune).

        gradient: time whole gradient evaluations on the gradient workspace (else forward
        steps on the forward workspace).  Returns {variant: ms per evaluation or per step}.
        """
        nv = self.variants
        ms = (ctypes.c_double * (max(nv, 0) + 1))()
        kind = B.PAT_WS_GRADIENT if gradient else B.PAT_WS_FORWARD
        ws = self.workspace(kind)
        with torch.cuda.device(self.device):
            B.check(B.lib().pat_plan_autotune(self._h, _ptr(ws), self.workspace_bytes(kind), ms, _stream(stream)),
                    "pat_plan_autotune")
        return {v: ms[v + 1] for v in range(-1, max(nv, 0))}

    def status(self, kind: int = B.PAT_WS_GRADIENT, stream=None) -> int:
        """pat_status of a cached workspace: PAT_STATUS_NONFINITE | PAT_STATUS_WAIT bits (synchronises)."""
        flag = ctypes.c_int(0)
        ws = self.workspace(kind)
        B.check(B.lib().pat_status(self._h, _ptr(ws), ctypes.byref(flag), _stream(stream)), "pat_status")
        return int(flag.value)

    def nonfinite(self, stream=None) -> bool:
        """True if the last objective on the gradient workspace met NaN/Inf (synchronises)."""
        return bool(self.status(B.PAT_WS_GRADIENT, stream) & B.PAT_STATUS_NONFINITE)



class Prior:
    """Ornstein-Uhlenbeck prior terms on an n x n grid (wraps pat_prior; Sec. 4.1.2).

    ``xi(v)``: Xi v; ``solve(b)``: Xi^{-1} b; ``eval(x, eta, sigma)``: the prior
    value sum_f 1/2 (x_f - eta_f)^T Xi^{-1} (x_f - eta_f) / sigma_f^2 and its
    gradient.  Fields are float32 CUDA tensors [nf][n][n].
    """

    def __init__(self, n: int, dx: float, tau: float, max_fields: int, device=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.n, self.max_fields = int(n), int(max_fields)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            B.check(B.lib().pat_prior_create(self.n, float(dx), float(tau), self.max_fields, ctypes.byref(h)),
                    "pat_prior_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                B.lib().pat_prior_destroy(h)
            except Exception:
                pass
            self._h = None

    def _shape(self, t, name):
        nf = int(t.shape[0])
        _f32(t, (nf, self.n, self.n), name, self.device)
        return nf

    def xi(self, v, stream=None):
        nf = self._shape(v, "v")
        out = torch.empty_like(v)
        with torch.cuda.device(self.device):
            B.check(B.lib().pat_prior_xi(self._h, _ptr(v), _ptr(out), nf, _stream(stream)), "pat_prior_xi")
        return out

    def solve(self, b, z=None, tol=1e-6, maxit=500, stream=None):
        """(Xi^{-1} b, iterations); z: warm start (overwritten with the solution)."""
        nf = self._shape(b, "b")
        warm = z is not None
        if z is None:
            z = torch.empty_like(b)
        it = ctypes.c_int(0)
        with torch.cuda.device(self.device):
            B.check(B.lib().pat_prior_solve(self._h, _ptr(b), _ptr(z), nf, float(tol), int(maxit), int(warm),
                                            ctypes.byref(it), _stream(stream)), "pat_prior_solve")
        return z, it.value

    def eval(self, x, eta, sigma, gscale=None, z=None, grad=None, tol=1e-6, maxit=500, stream=None):
        """(value, gradient added into ``grad`` (new zeros if None), z, iterations)."""
        nf = self._shape(x, "x")
        arr = lambda v: (ctypes.c_double * nf)(*[float(a) for a in v])
        warm = z is not None
        if z is None:
            z = torch.empty_like(x)
        if grad is None:
            grad = torch.zeros_like(x)
        J = torch.zeros((), dtype=torch.float64, device=self.device)
        it = ctypes.c_int(0)
        with torch.cuda.device(self.device):
            B.check(B.lib().pat_prior_eval(self._h, _ptr(x), nf, arr(eta), arr(sigma),
                                           arr(gscale) if gscale is not None else None, _ptr(z), _ptr(grad),
                                           _ptr(J), float(tol), int(maxit), int(warm), ctypes.byref(it),
                                           _stream(stream)), "pat_prior_eval")
        return float(J.item()), grad, z, it.value

def prolong(src, n_dst: int, stream=None):
    """Bilinear prolongation of fields [nb][n][n] to [nb][n_dst][n_dst] (pat_prolong)."""
    if src.dim() != 3 or src.shape[1] != src.shape[2]:
        raise ValueError("src must be [nb][n][n]")
    _f32(src, tuple(src.shape), "src", src.device)
    out = torch.empty((src.shape[0], int(n_dst), int(n_dst)), dtype=torch.float32, device=src.device)
    with torch.cuda.device(src.device):
        B.check(B.lib().pat_prolong(_ptr(src), _ptr(out), int(src.shape[0]), int(src.shape[1]), int(n_dst),
                                    _stream(stream)), "pat_prolong")
    return out


def time_interp(y, dt_src: float, dt_dst: float, nt_dst: int, stream=None):
    """Linear interpolation of traces [K][nt][m] to t = n dt_dst, n < nt_dst (pat_time_interp)."""
    if y.dim() != 3:
        raise ValueError("y must be [K][nt][m]")
    _f32(y, tuple(y.shape), "y", y.device)
    K, nts, m = (int(v) for v in y.shape)
    out = torch.empty((K, int(nt_dst), m), dtype=torch.float32, device=y.device)
    with torch.cuda.device(y.device):
        B.check(B.lib().pat_time_interp(_ptr(y), _ptr(out), K, nts, int(nt_dst), m, float(dt_src), float(dt_dst),
                                        _stream(stream)), "pat_time_interp")
    return out


@dataclass
class ReconConfig:
    """Parameters of pat_reconstruct (see include/pat.h)."""
    levels: tuple
    L: float
    dt_data: float
    nt_data: int
    sensors_xy: object
    K: int
    cfl: float = 0.3
    c_lo: float = 1350.0
    c_hi: float = 1750.0
    p0_lo: float = 0.0
    c_bg: float = 1500.0
    rho0: float = 1000.0
    pml_alpha: float = 2.0
    min_pml: int = 20
    mem: int = 20
    iters: int = 20
    max_halvings: int = 20
    ckpt_every: int = 32
    rtol: float = 1e-4
    alpha0: float = 0.1
    c1: float = 1e-4
    sigma_p0: float = 0.25
    autotune: bool = False
    # Ornstein-Uhlenbeck prior (Sec. 4.1.2): tau > 0 enables it
    prior_tau: float = 0.0
    prior_eta_c: float = 0.0
    prior_sigma_c: float = 0.0
    prior_eta_p0: float = 0.0
    prior_sigma_p0: float = 0.0
    persistent: bool = False   # forward sweeps as one persistent launch where the grid side has one


def _cfg_struct(cfg: ReconConfig, K: int, xy):
    lv = (ctypes.c_int * len(cfg.levels))(*[int(v) for v in cfg.levels])
    c_cfg = B.PatReconCfg(len(cfg.levels), lv, cfg.L, cfg.dt_data, cfg.nt_data, xy.shape[0],
                          xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), K, cfg.cfl, cfg.c_lo, cfg.c_hi,
                          cfg.p0_lo, cfg.c_bg, cfg.rho0, cfg.pml_alpha, cfg.min_pml, cfg.mem, cfg.iters,
                          cfg.max_halvings, cfg.ckpt_every, cfg.rtol, cfg.alpha0, cfg.c1, cfg.sigma_p0,
                          int(bool(cfg.autotune)), cfg.prior_tau, cfg.prior_eta_c, cfg.prior_sigma_c,
                          cfg.prior_eta_p0, cfg.prior_sigma_p0, int(bool(cfg.persistent)))
    return c_cfg, lv


def _rows(rep, rows):
    return [dict(level=r.level, it=r.iter, J=r.J, gnorm=r.gnorm, alpha=r.alpha, trials=r.trials, J_new=r.J_new,
                 ms=r.ms, Ec=r.Ec, Ep0=r.Ep0) for r in rows[:rep.count]]


def write_report_jsonl(rows, path, **fields):
    """Append one JSON line per L-BFGS iteration (level, iteration, J, |g|, step, trials, J after
    the step, wall ms, E_c, E_p0 as returned by reconstruct / reconstruct_batched) to path, each
    with the given extra fields (e.g. instance=3)."""
    with open(path, "a") as f:
        for r in rows:
            f.write(json.dumps(dict(fields, **r)) + "\n")


def reconstruct_batched(cfg: ReconConfig, instances, stream=None, max_report=4096):
    """Several reconstructions sharing cfg, solved together (pat_reconstruct_batched).

    ``instances``: list of dicts with device tensors ``y_meas`` [K][nt][m],
    ``w`` [K], ``c_init`` [N][N] and optional ``p0_init`` [K][N][N], ``c_true``
    [N][N] (E_c per iteration), ``p0_true`` [K][N][N] (E_p0 per iteration) and
    the targets ``ec_target`` / ``ep0_target`` (leave a level, the finest: stop,
    once every given target is reached).  Returns a list of (c, p0, report rows, status) and the
    total wall time in ms.
    """
    N = int(cfg.levels[-1])
    xy = np.ascontiguousarray(np.asarray(cfg.sensors_xy, dtype=np.float64))
    outs, structs, keep = [], [], []
    for ins in instances:
        ym, w = ins["y_meas"], ins["w"]
        K = int(ym.shape[0])
        dev = ym.device
        _f32(ym, (K, cfg.nt_data, xy.shape[0]), "y_meas", dev)
        _f32(w, (K,), "w", dev)
        c = ins["c_init"].detach().clone().contiguous()
        p0 = torch.zeros((K, N, N), dtype=torch.float32, device=dev) if ins.get("p0_init") is None else \
            ins["p0_init"].detach().clone().contiguous()
        _f32(c, (N, N), "c_init", dev)
        _f32(p0, (K, N, N), "p0_init", dev)
        rows = (B.PatIterReport * max_report)()
        rep = B.PatReport(max_report, 0, rows, 0, 0.0)
        keep.append((rows, rep))
        ct = ins.get("c_true")
        if ct is not None:
            _f32(ct, (N, N), "c_true", dev)
        pt = ins.get("p0_true")
        if pt is not None:
            _f32(pt, (K, N, N), "p0_true", dev)
        structs.append(B.PatInstance(ym.data_ptr(), w.data_ptr(), c.data_ptr(), p0.data_ptr(), K,
                                     ctypes.pointer(rep), ct.data_ptr() if ct is not None else None,
                                     float(ins.get("ec_target", 0.0)), pt.data_ptr() if pt is not None else None,
                                     float(ins.get("ep0_target", 0.0))))
        outs.append((c, p0))
    arr = (B.PatInstance * len(structs))(*structs)
    c_cfg, lv = _cfg_struct(cfg, 0, xy)
    dev = instances[0]["y_meas"].device
    with torch.cuda.device(dev):
        B.check(B.lib().pat_reconstruct_batched(ctypes.byref(c_cfg), len(structs), arr, _stream(stream)),
                "pat_reconstruct_batched")
    res = [(c, p0, _rows(rep, rows), int(rep.status)) for (c, p0), (rows, rep) in zip(outs, keep)]
    return res, float(keep[0][1].total_ms)


def reconstruct(cfg: ReconConfig, y_meas, w, c_init, p0_init=None, stream=None, max_report=4096):
    """Joint reconstruction (pat_reconstruct).  Returns (c, p0, report rows, status, total_ms).

    ``c_init``/``p0_init`` are device tensors on the finest level ([N][N] and
    [K][N][N]); they are copied, not modified.
    """
    N = int(cfg.levels[-1])
    K = int(cfg.K)
    dev = y_meas.device
    c = c_init.detach().clone().contiguous()
    p0 = torch.zeros((K, N, N), dtype=torch.float32, device=dev) if p0_init is None else \
        p0_init.detach().clone().contiguous()
    _f32(c, (N, N), "c_init", dev)
    _f32(p0, (K, N, N), "p0_init", dev)
    xy = np.ascontiguousarray(np.asarray(cfg.sensors_xy, dtype=np.float64))
    _f32(y_meas, (K, cfg.nt_data, xy.shape[0]), "y_meas", dev)
    _f32(w, (K,), "w", dev)
    c_cfg, lv = _cfg_struct(cfg, K, xy)
    rows = (B.PatIterReport * max_report)()
    rep = B.PatReport(max_report, 0, rows, 0, 0.0)
    with torch.cuda.device(dev):
        B.check(B.lib().pat_reconstruct(ctypes.byref(c_cfg), _ptr(y_meas), _ptr(w), _ptr(c), _ptr(p0),
                                        ctypes.byref(rep), _stream(stream)), "pat_reconstruct")
    return c, p0, _rows(rep, rows), int(rep.status), float(rep.total_ms)


def _fingerprint(cfg: ReconConfig, tensors, extra=None) -> str:
    """Hash of the configuration, the inputs and any extra JSON-able settings (targets) that a
    resumed run must share with the first."""
    h = hashlib.sha256()
    fields = {k: (np.asarray(v, dtype=np.float64).tolist() if k == "sensors_xy" else
                  [int(x) for x in v] if k == "levels" else v)
              for k, v in dataclasses.asdict(cfg).items()}
    h.update(json.dumps(fields, sort_keys=True).encode())
    h.update(json.dumps(extra).encode())
    for t in tensors:
        a = np.ascontiguousarray(t.detach().cpu().numpy())
        h.update(str(a.shape).encode())
        h.update(a.tobytes())
    return h.hexdigest()


_ROW_FIELDS = ("level", "it", "J", "gnorm", "alpha", "trials", "J_new", "ms", "Ec", "Ep0")


def reconstruct_batched_resumable(cfg: ReconConfig, instances, state_path, stop_after_level=None, stream=None,
                                  max_report=4096):
    """Batched reconstructions (as reconstruct_batched) that can stop after any multigrid level and
    continue later from a host file.

    The schedule runs one level per pat_reconstruct_batched call (levels=(N_l,)).  A level
    boundary is where the method itself ends one optimisation and starts the next from the
    prolonged point with an empty L-BFGS memory (Sec. 3.1), so the state there is every
    instance's iterate alone: no curvature pairs, and no random numbers (the reconstruction
    draws none).  After each level the state (levels done; every instance's c and p0 on that
    level's grid, report rows so far and status; the wall time; a fingerprint of cfg and of all
    inputs and targets) is written to ``state_path`` (an .npz, replaced atomically).  Called with
    an existing state file it checks the fingerprint (ValueError if cfg, an input or a target
    differs) and continues with the next level.  Every level starts from the same bilinear
    transfer (pat_prolong) that pat_reconstruct_batched applies between levels, the true c and
    p0 of E_c / E_p0 tracking are resampled from the finest grid as it does, and resampling onto
    the same grid inside a call is the identity, so with the kernel variants fixed (cfg.autotune
    off) the results are bit-identical to one pat_reconstruct_batched call over all levels.
    ``stop_after_level`` = l returns after level l (an interruption at a level boundary).

    ``instances``: as for reconstruct_batched, on the finest grid.  Returns (a list of (c, p0,
    report rows, status) per instance, total_ms, levels_done); c and p0 are on the grid of the
    last level done (the finest once levels_done == len(cfg.levels)).
    """
    levels = [int(v) for v in cfg.levels]
    N = levels[-1]
    inputs, cur = [], []
    for ins in instances:
        ym = ins["y_meas"]
        K, dev = int(ym.shape[0]), ym.device
        p0 = ins.get("p0_init")
        p0 = torch.zeros((K, N, N), dtype=torch.float32, device=dev) if p0 is None else p0
        _f32(ins["c_init"], (N, N), "c_init", dev)
        _f32(p0, (K, N, N), "p0_init", dev)
        inputs += [ym, ins["w"], ins["c_init"], p0] + [ins[k] for k in ("c_true", "p0_true") if ins.get(k) is not None]
        cur.append([ins["c_init"].detach().clone().contiguous(), p0.detach().clone().contiguous(), [], 0])
    targets = [[float(ins.get("ec_target", 0.0)), float(ins.get("ep0_target", 0.0)),
                ins.get("c_true") is not None, ins.get("p0_true") is not None] for ins in instances]
    fp = _fingerprint(cfg, inputs, extra=targets)
    done, total = 0, 0.0
    if os.path.exists(state_path):
        with np.load(state_path, allow_pickle=False) as z:
            meta = json.loads(str(z["meta"]))
            if meta["fingerprint"] != fp:
                raise ValueError(f"{state_path}: saved by a run with another configuration or other inputs")
            done, total = int(meta["levels_done"]), float(meta["total_ms"])
            for i, st in enumerate(cur):
                dev = instances[i]["y_meas"].device
                st[0] = torch.as_tensor(z[f"c{i}"], device=dev).contiguous()
                st[1] = torch.as_tensor(z[f"p0{i}"], device=dev).contiguous()
                st[2] = [dict(zip(_ROW_FIELDS, r)) for r in meta["rows"][i]]
                st[3] = int(meta["status"][i])
    last = len(levels) - 1 if stop_after_level is None else min(int(stop_after_level), len(levels) - 1)
    for li in range(done, last + 1):
        n_l = levels[li]
        lv = []
        for ins, (c, p0, _, _) in zip(instances, cur):
            d = {"y_meas": ins["y_meas"], "w": ins["w"],
                 "c_init": prolong(c.view(1, *c.shape), n_l, stream=stream)[0].contiguous(),
                 "p0_init": prolong(p0, n_l, stream=stream)}
            if ins.get("c_true") is not None:
                ct = ins["c_true"]
                d["c_true"] = prolong(ct.view(1, *ct.shape), n_l, stream=stream)[0].contiguous()
            if ins.get("p0_true") is not None:
                d["p0_true"] = prolong(ins["p0_true"], n_l, stream=stream)
            for k in ("ec_target", "ep0_target"):
                if k in ins:
                    d[k] = ins[k]
            lv.append(d)
        res, ms = reconstruct_batched(dataclasses.replace(cfg, levels=(n_l,)), lv, stream=stream,
                                      max_report=max_report)
        for st, (c, p0, rows, status) in zip(cur, res):
            for row in rows:
                row["level"] = li
            st[0], st[1] = c, p0
            st[2] = st[2] + rows
            st[3] = status if status != 0 else st[3]
        total += ms
        done = li + 1
        meta = {"fingerprint": fp, "levels_done": done, "levels": levels, "total_ms": total,
                "status": [st[3] for st in cur], "rows": [[[row[k] for k in _ROW_FIELDS] for row in st[2]] for st in cur]}
        arrays = {}
        for i, st in enumerate(cur):
            arrays[f"c{i}"] = st[0].cpu().numpy()
            arrays[f"p0{i}"] = st[1].cpu().numpy()
        buf = io.BytesIO()
        np.savez(buf, meta=np.array(json.dumps(meta)), **arrays)
        tmp = f"{state_path}.tmp{os.getpid()}"
        with open(tmp, "wb") as f:
            f.write(buf.getvalue())
        os.replace(tmp, state_path)
    return [tuple(st) for st in cur], total, done


def reconstruct_resumable(cfg: ReconConfig, y_meas, w, c_init, state_path, p0_init=None, stop_after_level=None,
                          stream=None, max_report=4096):
    """Joint reconstruction (as reconstruct) that can stop after any multigrid level and continue
    later from a host file: reconstruct_batched_resumable with one instance (pat_reconstruct is
    pat_reconstruct_batched with one instance), so bit-identical to one uninterrupted
    pat_reconstruct when the kernel variants are fixed.

    Returns (c, p0, report rows, status, total_ms, levels_done); c and p0 are on the grid of the
    last level done (the finest once levels_done == len(cfg.levels)).
    """
    ins = {"y_meas": y_meas, "w": w, "c_init": c_init}
    if p0_init is not None:
        ins["p0_init"] = p0_init
    res, total, done = reconstruct_batched_resumable(cfg, [ins], state_path, stop_after_level=stop_after_level,
                                                     stream=stream, max_report=max_report)
    c, p0, rows, status = res[0]
    return c, p0, rows, status, total, done
