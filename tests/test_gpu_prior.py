"""GPU Ornstein-Uhlenbeck prior (pat_prior_*) against the oracle's dense Xi (Sec. 4.1.2).

Xi v is an exact FFT convolution (FP32: 1e-5 relative); Xi^{-1} b comes from
preconditioned CG to a relative residual of 1e-6 (1e-4 relative against the
oracle's Cholesky solve; a warm start needs fewer iterations than a cold one);
prior values and gradients to 1e-4.  On the
headline grid (256 x 256, dx = 0.1 mm, tau = 1.5 mm) Xi v is checked at
sampled pixels against rows of the oracle's Xi, and the solve by its residual.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("n,dx,tau,nf", [(24, 1e-4, 1.5e-3, 3), (40, 2e-4, 1.5e-3, 2), (37, 4e-4, 6e-4, 1)])
def test_xi_and_solve_match_dense(n, dx, tau, nf):
    from oracle.prior import OUPrior
    from paper_2505_08482_gb300.solver import Prior
    rng = np.random.default_rng(n)
    v = rng.standard_normal((nf, n, n))
    pr = OUPrior((n, n), dx, tau)
    gp = Prior(n, dx, tau, max_fields=4)
    xv = gp.xi(_dev(v)).cpu().numpy()
    for f in range(nf):
        assert _rel(xv[f], (pr.xi @ v[f].ravel()).reshape(n, n)) <= 1e-5
    z, it = gp.solve(_dev(v), tol=1e-6, maxit=500)
    assert 0 < it < 500
    zo = pr.solve(v)
    assert _rel(z.cpu().numpy(), zo) <= 1e-4
    # warm start at the solution: its FP32 residual (about 1e-5) still needs some iterations
    z2, it2 = gp.solve(_dev(v), z=z.clone(), tol=1e-6, maxit=500)
    assert it2 < it and _rel(z2.cpu().numpy(), zo) <= 1e-4


def test_eval_value_and_gradient():
    from oracle.prior import OUPrior, prior_value_grad
    from paper_2505_08482_gb300.solver import Prior
    n, dx, tau = 32, 2e-4, 1.5e-3
    rng = np.random.default_rng(7)
    p0 = rng.uniform(0.0, 1.0, (2, n, n))
    c = 1525.0 + 40.0 * rng.standard_normal((n, n))
    J, gp0, gc = prior_value_grad(OUPrior((n, n), dx, tau), p0, c, 0.5, 0.25, 1525.0, 62.5)
    gp = Prior(n, dx, tau, max_fields=3)
    x = _dev(np.concatenate([p0, c[None]]))
    base = torch.ones_like(x)
    val, grad, z, it = gp.eval(x, [0.5, 0.5, 1525.0], [0.25, 0.25, 62.5], gscale=[0.25, 0.25, 100.0],
                               grad=base.clone(), tol=1e-6)
    assert val == pytest.approx(J, rel=1e-4)
    g = grad.cpu().numpy() - 1.0
    assert _rel(g[:2] / 0.25, gp0) <= 1e-4 and _rel(g[2] / 100.0, gc) <= 1e-4
    # value only, warm: same value, gradient untouched
    val2, grad2, _, it2 = gp.eval(x, [0.5, 0.5, 1525.0], [0.25, 0.25, 62.5], z=z, grad=base.clone(), tol=1e-6)
    assert val2 == pytest.approx(J, rel=1e-4) and it2 < it


def test_headline_grid_sampled():
    from oracle.prior import pixel_points, unit_covariance
    from paper_2505_08482_gb300.solver import Prior
    import pat_synth as ps
    n, dx, tau = 256, 1e-4, 1.5e-3
    w = ps.workload("vessels256", 0)
    v = np.concatenate([w.p0_true, (w.c_true - 1525.0)[None] / 62.5])          # 9 fields
    gp = Prior(n, dx, tau, max_fields=9)
    xv = gp.xi(_dev(v)).cpu().numpy()
    rows = np.array([0, 255, 256 * 128 + 77, 256 * 255 + 3, 256 * 40 + 200, n * n - 1])
    R = unit_covariance(pixel_points((n, n), dx), tau, rows)
    for f in (0, 4, 8):
        ref = R @ v[f].ravel()
        np.testing.assert_allclose(xv[f].ravel()[rows], ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())
    z, it = gp.solve(_dev(v), tol=1e-6, maxit=500)
    assert it < 500
    res = gp.xi(z).cpu().numpy() - v
    for f in range(9):
        assert np.linalg.norm(res[f]) <= 1e-4 * np.linalg.norm(v[f])


def test_reconstruction_with_prior_matches_oracle():
    from oracle.forward import forward
    from oracle.grid import make_grid
    from oracle.multigrid import reconstruct as oracle_recon
    from oracle.sensors import sensor_matrix
    from paper_2505_08482_gb300.solver import ReconConfig, reconstruct
    import pat_synth as ps
    w = ps.workload("plain64", 2)
    g = make_grid(64, w.dx, 300, c_ref=1750.0)
    y = ps.add_noise(forward(g, w.c_true, w.p0_true, sensor_matrix(g, w.sensors)), ps.rng_for(102))
    wt = ps.noise_weights(y)
    lo, hi = w.c_true.min(), w.c_true.max()
    prior = dict(tau=1.5e-3, eta_c=0.5 * (lo + hi), sigma_c=0.25 * (hi - lo), eta_p0=0.5 * w.p0_true.max(),
                 sigma_p0=0.25 * w.p0_true.max())
    T = (g.nt - 1) * g.dt
    _, _, hist = oracle_recon([32, 64], 64 * w.dx, T, w.sensors, y, g.dt, wt, prior["eta_c"], (1350.0, 1750.0),
                              iters=3, mem=20, rtol=0.0, prior=prior)
    cfg = ReconConfig(levels=(32, 64), L=64 * w.dx, dt_data=g.dt, nt_data=g.nt, sensors_xy=w.sensors, K=1,
                      mem=20, iters=3, rtol=0.0, ckpt_every=32, prior_tau=prior["tau"], prior_eta_c=prior["eta_c"],
                      prior_sigma_c=prior["sigma_c"], prior_eta_p0=prior["eta_p0"],
                      prior_sigma_p0=prior["sigma_p0"])
    c_g, p0_g, rows, status, ms = reconstruct(cfg, _dev(y), _dev(wt), _dev(np.full((64, 64), prior["eta_c"])))
    ref = [(h["level"], e) for h in hist for e in h["result"].history]
    assert len(rows) == len(ref)
    for r, (lv, e) in zip(rows, ref):
        assert r["level"] == lv and r["it"] == e["it"]
        assert abs(r["J"] - e["J"]) <= 1e-3 * e["J"]
        assert abs(r["gnorm"] - e["gnorm"]) <= 1e-3 * e["gnorm"]
        assert r["alpha"] == e["alpha"] and r["trials"] == e["trials"]
