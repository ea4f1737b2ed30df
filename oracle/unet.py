"""Reference U-Net of the learned warm start (oracle, plain PyTorch on the CPU).

Test infrastructure only.  The paper has no network; this module states the
architecture of the library's U-Net with plain library primitives (conv2d,
max pooling, nearest upsampling, ReLU) so that the GPU forward pass and its
parameter gradients can be compared with it.  Parameters use the library's
flat layout: for every convolution in forward order (encoder a/b per level,
decoder a/b per level from the deepest, final 1x1), weights [cout][k*k][cin]
then bias [cout]; tap t of a 3x3 kernel is at (dy, dx) = (t // 3 - 1, t % 3 - 1)
(cross-correlation).  The input has in_ch channels zero-padded to a multiple
of 8.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as Fn


def pad8(c: int) -> int:
    return (c + 7) // 8 * 8


def conv_specs(levels: int, base: int, in_ch: int):
    """(cin, cout, k) of every convolution in forward order."""
    specs = []
    cprev = pad8(in_ch)
    for l in range(levels):
        ch = base << l
        specs += [(cprev, ch, 3), (ch, ch, 3)]
        cprev = ch
    for l in range(levels - 2, -1, -1):
        ch = base << l
        specs += [(cprev + ch, ch, 3), (ch, ch, 3)]
        cprev = ch
    specs.append((cprev, 1, 1))
    return specs


def param_count(levels, base, in_ch):
    return sum(co * k * k * ci + co for ci, co, k in conv_specs(levels, base, in_ch))


def init_params(levels, base, in_ch, rng) -> np.ndarray:
    """He-normal weights (zero on the padding input channels), zero biases."""
    out = []
    for i, (ci, co, k) in enumerate(conv_specs(levels, base, in_ch)):
        w = rng.standard_normal((co, k * k, ci)) * np.sqrt(2.0 / (k * k * ci))
        if i == 0:
            w[:, :, in_ch:] = 0.0
        out += [w.ravel(), np.zeros(co)]
    return np.concatenate(out)


def _unpack(params, levels, base, in_ch, dtype):
    p = torch.as_tensor(np.asarray(params), dtype=dtype) if not torch.is_tensor(params) else params
    convs, o = [], 0
    for ci, co, k in conv_specs(levels, base, in_ch):
        n = co * k * k * ci
        w = p[o:o + n].reshape(co, k * k, ci).permute(0, 2, 1).reshape(co, ci, k, k)
        o += n
        b = p[o:o + co]
        o += co
        convs.append((w, b))
    return convs


def forward(params, x, levels, base, in_ch, dtype=torch.float64):
    """x: [B][in_ch][H][W] -> [B][H][W]."""
    convs = _unpack(params, levels, base, in_ch, dtype)
    x = torch.as_tensor(np.asarray(x), dtype=dtype) if not torch.is_tensor(x) else x
    B, C, H, W = x.shape
    h = torch.zeros((B, pad8(in_ch), H, W), dtype=dtype)
    h[:, :C] = x
    it = iter(convs)

    def conv(t, relu=True):
        w, b = next(it)
        pad = (w.shape[-1] - 1) // 2
        y = Fn.conv2d(t, w, b, padding=pad)
        return Fn.relu(y) if relu else y

    skips = []
    for l in range(levels):
        h = conv(conv(h))
        if l < levels - 1:
            skips.append(h)
            h = Fn.max_pool2d(h, 2)
    for l in range(levels - 2, -1, -1):
        h = Fn.interpolate(h, scale_factor=2, mode="nearest")
        h = torch.cat([h, skips[l]], dim=1)
        h = conv(conv(h))
    return conv(h, relu=False)[:, 0]


def loss_and_grad(params, x, target, levels, base, in_ch, dtype=torch.float64):
    """MSE loss mean((out - target)^2) and its gradient with respect to the flat parameters."""
    p = torch.as_tensor(np.asarray(params), dtype=dtype).clone().requires_grad_(True)
    out = forward(p, x, levels, base, in_ch, dtype)
    t = torch.as_tensor(np.asarray(target), dtype=dtype)
    loss = torch.mean((out - t) ** 2)
    loss.backward()
    return float(loss.detach()), p.grad.numpy().copy()
