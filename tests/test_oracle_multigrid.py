"""Coarse-to-fine reconstruction with the oracle on a tiny problem (Sec. 3.1)."""
import numpy as np

from oracle import forward as F
from oracle.grid import make_grid
from oracle.metrics import relative_error
from oracle.multigrid import reconstruct
from oracle.sensors import sensor_matrix
import pat_synth as ps


def test_two_level_reconstruction_improves_both_unknowns():
    w = ps.workload("tiny16", 0)
    g = make_grid(16, w.dx, 120, c_ref=1750.0, min_pml=8)
    S = sensor_matrix(g, w.sensors)
    y = F.forward(g, w.c_true, w.p0_true, S)
    y = ps.add_noise(y, ps.rng_for(11))
    wt = ps.noise_weights(y)
    T = (g.nt - 1) * g.dt
    c_init = 0.5 * (w.c_true.min() + w.c_true.max())
    seen = []
    p0, c, hist = reconstruct([8, 16], 16 * w.dx, T, w.sensors, y, g.dt, wt, c_init, (1350.0, 1750.0),
                              iters=6, min_pml=8, callback=lambda l, i, x, J: seen.append((l, J)))
    for h in hist:
        Js = [e["J"] for e in h["result"].history]
        assert all(b <= a for a, b in zip(Js, Js[1:]))
    assert relative_error(w.p0_true, p0) < 100.0
    assert np.all(p0 >= 0.0) and np.all((c >= 1350.0) & (c <= 1750.0))
    assert relative_error(w.c_true, c) < relative_error(w.c_true, np.full_like(c, c_init)) + 1e-9
    assert len(seen) > 0
