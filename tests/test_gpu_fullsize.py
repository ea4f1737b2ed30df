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
