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


def test_each_level_equals_a_fresh_solve_from_the_prolonged_point():
    """The level loop composed from its parts: for every level, a projected L-BFGS started afresh
    (no curvature pairs) from the prolongation of the previous level's result, on a grid and data
    built independently for that level (dx = L/N, dt from the CFL at U_c, Nt = round(T/dt) + 1,
    data interpolated to that time grid), must take exactly the steps the loop recorded.  A wrong
    per-level time grid, data interpolation or prolongation, or curvature pairs carried over from
    the coarser level, changes the first iteration."""
    from oracle.adjoint import adjoint_grad, objective
    from oracle.lbfgs import projected_lbfgs
    from oracle.multigrid import level_nt, prolong, time_interp
    w = ps.workload("tiny16", 1)
    g = make_grid(16, w.dx, 100, c_ref=1750.0, min_pml=8)
    y = ps.add_noise(F.forward(g, w.c_true, w.p0_true, sensor_matrix(g, w.sensors)), ps.rng_for(12))
    wt = ps.noise_weights(y)
    T, L, K = (g.nt - 1) * g.dt, 16 * w.dx, w.p0_true.shape[0]
    levels, iters = [8, 12, 16], 4
    p0, c, hist = reconstruct(levels, L, T, w.sensors, y, g.dt, wt, 1500.0, (1350.0, 1750.0), iters=iters, mem=5,
                              min_pml=8, rtol=0.0)
    x_prev = None
    for li, (nl, h) in enumerate(zip(levels, hist)):
        gl = make_grid(nl, L / nl, 1, c_ref=1750.0, min_pml=8)
        gl.nt = level_nt(T, gl.dt)
        assert h["nt"] == gl.nt and h["n"] == nl
        S = sensor_matrix(gl, w.sensors)
        yl = time_interp(y, g.dt, gl.dt, gl.nt)
        npx = nl * nl
        if x_prev is None:
            x0 = np.concatenate([np.zeros(K * npx), np.full(npx, 1500.0)])
        else:
            pp, cc = x_prev
            x0 = np.concatenate([prolong(pp, nl).ravel(), prolong(cc, nl).ravel()])
        unpack = lambda x: (x[:K * npx].reshape(K, nl, nl), x[K * npx:].reshape(nl, nl))

        def fun(x):
            pp_, cc_ = unpack(x)
            return objective(gl, cc_, pp_, S, yl, wt)[0]

        def fun_grad(x):
            pp_, cc_ = unpack(x)
            J, gp, gc = adjoint_grad(gl, cc_, pp_, S, yl, wt)
            return J, np.concatenate([gp.ravel(), gc.ravel()])

        lo = np.concatenate([np.zeros(K * npx), np.full(npx, 1350.0)])
        hi = np.concatenate([np.full(K * npx, np.inf), np.full(npx, 1750.0)])
        sc = np.concatenate([np.full(K * npx, 0.25), np.full(npx, 100.0)])
        ref = projected_lbfgs(fun, fun_grad, x0, lo, hi, sc, mem=5, max_iter=iters, rtol=0.0)
        got = h["result"]
        assert len(got.history) == len(ref.history)
        for a, b in zip(got.history, ref.history):
            assert a["J"] == b["J"] and a["alpha"] == b["alpha"]
        np.testing.assert_array_equal(got.x, ref.x)
        x_prev = unpack(got.x)
