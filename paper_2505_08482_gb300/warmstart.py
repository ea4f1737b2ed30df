"""Learned warm start: a U-Net that proposes the initial speed of sound.

Inputs are the K back-projected images BP_k = A_{c0}^T y_k (the adjoint of
the forward operator at a constant speed of sound c0, computed by the
library's adjoint kernels through pat_vjp), normalised by their common peak;
the target is (c_true - c0) / c_scale.  The network runs in the library's
BF16 tensor-core kernels (pat_unet_*); the plain iterative reconstruction
remains the fallback and the arbiter of the error.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _binding as B
from .solver import _ptr, _stream


class UNet:
    """Handle of a pat_unet (levels, base width, input channels, image size, max batch)."""

    def __init__(self, levels=4, base=32, in_ch=4, H=128, W=128, max_batch=32, device=None):
        self.levels, self.base, self.in_ch, self.H, self.W, self.max_batch = levels, base, in_ch, H, W, max_batch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            B.check(B.lib().pat_unet_create(ctypes.byref(h), levels, base, in_ch, H, W, max_batch), "pat_unet_create")
        self._h = h
        self.nparam = int(B.lib().pat_unet_param_count(h))
        self._loss = torch.zeros((), dtype=torch.float64, device=self.device)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                B.lib().pat_unet_destroy(h)
            except Exception:
                pass
            self._h = None

    @property
    def gemm_path(self) -> int:
        return getattr(self, "_gemm_path", 1)

    @gemm_path.setter
    def gemm_path(self, path: int):
        """1 (default): tcgen05 / TMEM / TMA; 0: warp-level tensor cores, mma.sync (pat_unet_set_gemm_path)."""
        B.check(B.lib().pat_unet_set_gemm_path(self._h, int(path)), "pat_unet_set_gemm_path")
        self._gemm_path = int(path)

    def status(self, stream=None) -> int:
        """PAT_STATUS_TC05 if a bounded wait of a tcgen05 GEMM gave up (synchronises)."""
        flag = ctypes.c_int(0)
        B.check(B.lib().pat_unet_status(self._h, ctypes.byref(flag), _stream(stream)), "pat_unet_status")
        return int(flag.value)

    def set_params(self, params, stream=None):
        p = torch.as_tensor(np.asarray(params, dtype=np.float32), device=self.device).contiguous()
        if p.numel() != self.nparam:
            raise ValueError(f"expected {self.nparam} parameters, got {p.numel()}")
        B.check(B.lib().pat_unet_set_params(self._h, _ptr(p), _stream(stream)), "pat_unet_set_params")
        torch.cuda.current_stream(self.device).synchronize()

    def get_params(self, stream=None) -> torch.Tensor:
        p = torch.empty(self.nparam, dtype=torch.float32, device=self.device)
        B.check(B.lib().pat_unet_get_params(self._h, _ptr(p), _stream(stream)), "pat_unet_get_params")
        return p

    def _check_in(self, x):
        if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous() or x.dim() != 4 or \
                tuple(x.shape[1:]) != (self.in_ch, self.H, self.W) or not 1 <= x.shape[0] <= self.max_batch:
            raise ValueError("input must be a contiguous float32 CUDA tensor [B][in_ch][H][W], B <= max_batch")

    def forward(self, x, stream=None) -> torch.Tensor:
        self._check_in(x)
        out = torch.empty((x.shape[0], self.H, self.W), dtype=torch.float32, device=self.device)
        B.check(B.lib().pat_unet_forward(self._h, _ptr(x), int(x.shape[0]), _ptr(out), _stream(stream)),
                "pat_unet_forward")
        return out

    def grads(self, x, target, stream=None):
        self._check_in(x)
        g = torch.empty(self.nparam, dtype=torch.float32, device=self.device)
        B.check(B.lib().pat_unet_grads(self._h, _ptr(x), _ptr(target.contiguous()), int(x.shape[0]), _ptr(g),
                                       _ptr(self._loss), _stream(stream)), "pat_unet_grads")
        return float(self._loss.item()), g

    def train_step(self, x, target, lr, stream=None) -> torch.Tensor:
        """One Adam step; returns the loss as a device scalar (no synchronisation)."""
        self._check_in(x)
        loss = torch.empty((), dtype=torch.float64, device=self.device)
        B.check(B.lib().pat_unet_train_step(self._h, _ptr(x), _ptr(target.contiguous()), int(x.shape[0]),
                                            ctypes.c_float(lr), _ptr(loss), _stream(stream)), "pat_unet_train_step")
        return loss


def back_projection(plan, y, c0: float = 1500.0) -> torch.Tensor:
    """BP_k = A_{c0}^T y_k for y [K][nt][m] on a plan: adjoint at constant c0 (pat_vjp)."""
    n, K = plan.n, plan.K
    c = torch.full((n, n), float(c0), dtype=torch.float32, device=plan.device)
    z = torch.zeros((K, n, n), dtype=torch.float32, device=plan.device)
    plan.forward(c, z, keep_checkpoints=True)
    bp, _ = plan.vjp(c, z, y.contiguous())
    return bp


def normalise_bp(bp: torch.Tensor) -> torch.Tensor:
    """Scale the K images of one sample by their common peak (|.|max)."""
    s = bp.abs().amax(dim=(-3, -2, -1), keepdim=True).clamp_min(1e-30)
    return bp / s


# ---------------------------------------------------------------------------
# data, training and evaluation of the warm start

class PairGenerator:
    """Solver-generated training pairs (back-projection stack, scaled true c).

    One batched forward plan evaluates the data of ``batch`` instances at
    their true c; a second batched plan (store-all history, so the adjoint
    needs no recompute) back-projects the noisy data at the constant c0.
    """

    def __init__(self, n=128, K=4, M=256, nt=600, batch=64, dx=1e-4, c_hi=1750.0, c0=1500.0, c_scale=100.0,
                 device=None):
        import pat_synth as ps
        from .solver import GridSpec, Plan, pml_auto
        self.n, self.K, self.M, self.nt, self.batch = n, K, M, nt, batch
        self.c0, self.c_scale = c0, c_scale
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.gs = GridSpec(n=n, pml=pml_auto(n), dx=dx, dt=0.3 * dx / c_hi, nt=nt, c_ref=c_hi)
        self.sensors = ps.circle_sensors(n, M, dx)
        self.fwd = Plan(self.gs, self.sensors, [K] * batch, ckpt_every=nt, device=self.device)
        self.bp = Plan(self.gs, self.sensors, [K] * batch, ckpt_every=nt, device=self.device)

    def make(self, seeds, keep_data=False):
        """Inputs [B][K][n][n], targets [B][n][n] (and the raw data if keep_data) for the seeds."""
        import pat_synth as ps
        dev = self.device
        X, T, raw = [], [], []
        for b0 in range(0, len(seeds), self.batch):
            sb = list(seeds[b0:b0 + self.batch])
            pad = self.batch - len(sb)
            cs, p0s = [], []
            for s in sb:
                c, p0 = ps.warmstart_sample(self.n, self.K, s)
                cs.append(c)
                p0s.append(p0)
            for _ in range(pad):   # fill a partial batch with copies (discarded)
                cs.append(cs[-1])
                p0s.append(p0s[-1])
            c_t = torch.as_tensor(np.stack(cs), dtype=torch.float32, device=dev)
            p0_t = torch.as_tensor(np.concatenate(p0s), dtype=torch.float32, device=dev)
            y = self.fwd.forward(c_t, p0_t)
            gen = torch.Generator(device=dev)
            gen.manual_seed(int(sb[0]) * 7919 + 17)
            yn, w = ps.add_noise_torch(y, gen)
            cc = torch.full_like(c_t, self.c0)
            z = torch.zeros_like(p0_t)
            self.bp.forward(cc, z, keep_checkpoints=True)
            bp, _ = self.bp.vjp(cc, z, yn)
            bp = normalise_bp(bp.reshape(self.batch, self.K, self.n, self.n))
            nb = len(sb)
            X.append(bp[:nb].clone())
            T.append(((c_t[:nb] - self.c0) / self.c_scale).clone())
            if keep_data:
                for j in range(nb):
                    raw.append(dict(y_meas=yn[j * self.K:(j + 1) * self.K].clone(),
                                    w=w[j * self.K:(j + 1) * self.K].float().clone(),
                                    c_true=c_t[j].clone(), p0_true=p0_t[j * self.K:(j + 1) * self.K].clone()))
        return torch.cat(X), torch.cat(T), raw


def train(net: UNet, X, T, epochs=10, batch=32, lr=1e-3, seed=0, log_every=0):
    """Adam on shuffled mini-batches; returns the mean loss of every epoch."""
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    n = X.shape[0]
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g)
        losses = []
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch].to(X.device)
            xb = X.index_select(0, idx).contiguous()
            tb = T.index_select(0, idx).contiguous()
            losses.append(net.train_step(xb, tb, lr * (0.5 if ep >= 0.7 * epochs else 1.0)))
        hist.append(float(torch.stack(losses).mean().item()))
        if log_every and (ep + 1) % log_every == 0:
            print(f"epoch {ep + 1}: loss {hist[-1]:.5f}", flush=True)
    return hist


def predict_c(net: UNet, X, c0=1500.0, c_scale=100.0, bounds=(1350.0, 1750.0), batch=None):
    """Initial speed of sound c0 + c_scale * U-Net(X), clipped to the bounds."""
    batch = batch or net.max_batch
    outs = []
    for b0 in range(0, X.shape[0], batch):
        xb = X[b0:b0 + batch].contiguous()
        outs.append(net.forward(xb))
    return (c0 + c_scale * torch.cat(outs)).clamp(*bounds)


def relative_error(c, c_true):
    """E_c = 100 ||c - c_true|| / ||c_true|| per sample (Eq. RelativeError)."""
    d = (c - c_true).flatten(1).double()
    return 100.0 * d.norm(dim=1) / c_true.flatten(1).double().norm(dim=1)


def init_params(levels, base, in_ch, seed=0) -> np.ndarray:
    """He-normal weights (zero on the padding input channels), zero biases, in the library's layout."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pad8 = lambda c: (c + 7) // 8 * 8
    specs, cprev = [], pad8(in_ch)
    for l in range(levels):
        ch = base << l
        specs += [(cprev, ch, 3), (ch, ch, 3)]
        cprev = ch
    for l in range(levels - 2, -1, -1):
        ch = base << l
        specs += [(cprev + ch, ch, 3), (ch, ch, 3)]
        cprev = ch
    specs.append((cprev, 1, 1))
    out = []
    for i, (ci, co, k) in enumerate(specs):
        w = rng.standard_normal((co, k * k, ci)) * np.sqrt(2.0 / (k * k * ci))
        if i == 0:
            w[:, :, in_ch:] = 0.0
        out += [w.ravel(), np.zeros(co)]
    return np.concatenate(out).astype(np.float32)


def iterations_to(rows, target, nlevels, ep0_target=None):
    """(iterations over all levels, ms) until E_c <= target (and E_p0 <= ep0_target if given) on the
    finest level, or (None, None)."""
    its, ms = 0, 0.0
    for r in rows:
        its += 1
        ms += r["ms"]
        if r["level"] == nlevels - 1 and 0 <= r["Ec"] <= target and (
                ep0_target is None or 0 <= r.get("Ep0", -1.0) <= ep0_target):
            return its, ms
    return None, None
