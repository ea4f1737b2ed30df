"""Pins of the reference U-Net: convolution convention by direct sums, gradients by finite differences."""
import numpy as np
import torch

from oracle import unet as U


def test_conv_tap_convention_matches_direct_sum():
    rng = np.random.default_rng(0)
    ci, co, H, W = 3, 2, 5, 6
    x = rng.standard_normal((1, ci, H, W))
    w = rng.standard_normal((co, 9, ci))          # library layout [cout][tap][cin]
    b = rng.standard_normal(co)
    wt = torch.as_tensor(w).permute(0, 2, 1).reshape(co, ci, 3, 3)
    got = torch.nn.functional.conv2d(torch.as_tensor(x), wt, torch.as_tensor(b), padding=1).numpy()
    ref = np.zeros((1, co, H, W))
    for o in range(co):
        for y in range(H):
            for xx in range(W):
                s = b[o]
                for t in range(9):
                    yy, xs = y + t // 3 - 1, xx + t % 3 - 1
                    if 0 <= yy < H and 0 <= xs < W:
                        s += np.dot(w[o, t], x[0, :, yy, xs])
                ref[0, o, y, xx] = s
    assert np.abs(got - ref).max() < 1e-12


def test_param_count_and_layout():
    specs = U.conv_specs(4, 32, 4)
    assert specs[0] == (8, 32, 3) and specs[-1] == (32, 1, 1)
    assert specs[8] == (256 + 128, 128, 3)
    assert len(specs) == 15
    assert U.param_count(4, 32, 4) == sum(co * k * k * ci + co for ci, co, k in specs)


def test_unet_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    levels, base, in_ch = 2, 8, 2
    p = U.init_params(levels, base, in_ch, rng)
    p[-1] = 0.3                                     # nonzero final bias
    x = rng.standard_normal((2, in_ch, 8, 8))
    t = rng.standard_normal((2, 8, 8))
    L, g = U.loss_and_grad(p, x, t, levels, base, in_ch)
    for _ in range(4):
        d = rng.standard_normal(p.shape)
        d[:base * 9 * 8][np.tile(np.arange(8) >= in_ch, base * 9)] = 0.0   # padding weights stay zero
        h = 1e-6
        Lp = U.loss_and_grad(p + h * d, x, t, levels, base, in_ch)[0]
        Lm = U.loss_and_grad(p - h * d, x, t, levels, base, in_ch)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - np.dot(g, d)) <= 1e-6 * max(1.0, abs(fd))
