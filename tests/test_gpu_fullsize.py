"""Full-size parity at the benchmark workload (256 x 256 domain, Ng 300, K = 8, M = 512, Nt = 1800).

The oracle cannot step 1800 steps of 8 x 300^2 in seconds, but for a
homogeneous medium at the reference speed without absorption the scheme is
exact in time (closed form p^n = F^-1[cos(c |k| n dt) F p0], pinned on the
CPU), so the oracle evaluates sampled time steps one by one.  The gradient at
full size is checked by the adjoint identity and by finite differences in
tests/test_gpu_autograd.py.
"""
import numpy as np
import pytest

import pat_synth as ps
from tests._problems import grid_params, oracle_grid, gpu_plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_fullsize_traces_match_closed_form_samples(variant):
    # every fixed-size variant the benchmark's autotuner may pick
    from oracle.sensors import sensor_matrix
    w = ps.workload("vessels256", 0)
    gp = grid_params(256, 1800, pml_alpha=0.0, c_hi=1500.0)
    g = oracle_grid(gp)
    S = sensor_matrix(g, w.sensors)
    plan = gpu_plan(gp, w.sensors, 8, ckpt_every=32)
    if variant >= plan.variants:
        pytest.skip("no such variant for this grid side")
    plan.variant = variant
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    y = plan.forward(f(np.full((256, 256), 1500.0)), f(w.p0_true)).cpu().numpy()
    kabs = np.sqrt(g.KX ** 2 + g.KY ** 2)
    P0 = np.fft.fft2(g.pad(w.p0_true), axes=(-2, -1))
    num, den = 0.0, 0.0
    for n in (0, 1, 250, 600, 1200, 1799):
        pn = np.real(np.fft.ifft2(np.cos(1500.0 * kabs * n * g.dt) * P0, axes=(-2, -1)))
        ex = np.stack([S @ pn[k].ravel() for k in range(8)])
        num += np.sum((y[:, n] - ex) ** 2)
        den += np.sum(ex ** 2)
        assert np.abs(y[:, n] - ex).max() <= 1e-4 * np.abs(ex).max() + 1e-6 * np.abs(y).max()
    assert np.sqrt(num / den) <= 1e-4


def test_fullsize_heterogeneous_traces_match_the_oracle_on_sampled_data_sets():
    """The benchmark's grid, batch and kernel variant with its heterogeneous speed of sound:
    traces are causal, so the first 300 samples of data sets 0 and 7 of the full run
    (K = 8, Nt = 1800) equal an oracle run of 300 steps of that data set alone."""
    from oracle import forward as F
    from oracle.sensors import sensor_matrix
    w = ps.workload("vessels256", 0)
    plan = gpu_plan(grid_params(256, 1800), w.sensors, 8, ckpt_every=32)
    plan.variant = 0
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    y = plan.forward(f(w.c_true), f(w.p0_true)).cpu().numpy()
    ns = 300
    g = oracle_grid(grid_params(256, ns))
    S = sensor_matrix(g, w.sensors)
    for k in (0, 7):
        ref = F.forward(g, w.c_true, w.p0_true[k:k + 1], S)[0]
        assert np.abs(ref).max() > 0.1                     # the waves have reached the sensors
        err = np.linalg.norm(y[k, :ns] - ref) / np.linalg.norm(ref)
        assert err <= 1e-4, (k, err)


def test_fullsize_vjp_matches_the_oracle_for_a_source_in_the_first_samples():
    """The full reverse sweep of the benchmark's configuration (K = 8, Nt = 1800, s = 32
    checkpoints, recompute stream) with an adjoint source that is zero after the first 150
    samples and outside data sets 0 and 7: the adjoint stays exactly zero until then, so the
    result is the gradient of the 150-step problem of those two data sets, which the oracle
    computes (adjoint source r = ybar through y_meas = f(x) - ybar, w = 1)."""
    from paper_2505_08482_gb300 import _binding as B
    from oracle import forward as F
    from oracle.adjoint import adjoint_grad
    from oracle.sensors import sensor_matrix
    w = ps.workload("vessels256", 0)
    plan = gpu_plan(grid_params(256, 1800), w.sensors, 8, ckpt_every=32)
    plan.variant = 0
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    ns, ks = 150, [0, 7]
    p0 = 0.5 * w.p0_true
    ybar = np.zeros((8, 1800, w.m))
    ybar[ks, :ns] = ps.rng_for(7).standard_normal((2, ns, w.m))
    c, p0d = f(w.c_true), f(p0)
    plan.forward(c, p0d, keep_checkpoints=True)
    gp, gc = plan.vjp(c, p0d, f(ybar))
    gp, gc = gp.cpu().numpy(), gc.cpu().numpy()
    assert plan.workspace_bytes(B.PAT_WS_GRADIENT) > 0
    assert np.all(gp[[1, 2, 3, 4, 5, 6]] == 0.0)
    g = oracle_grid(grid_params(256, ns))
    S = sensor_matrix(g, w.sensors)
    y_o = F.forward(g, w.c_true, p0[ks], S)
    _, gp_o, gc_o = adjoint_grad(g, w.c_true, p0[ks], S, y_o - ybar[ks, :ns], np.ones(2))
    for j, k in enumerate(ks):
        assert np.linalg.norm(gp[k] - gp_o[j]) <= 1e-3 * np.linalg.norm(gp_o[j]), k
    assert np.linalg.norm(gc - gc_o) <= 1e-3 * np.linalg.norm(gc_o)
