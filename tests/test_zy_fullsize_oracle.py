"""Full-size parity against the oracle on sampled outputs (256 x 256 domain, Ng 300, K = 8,
M = 512, Nt = 1800, s = 32: the benchmark's grid, batch and kernel variant).

The oracle cannot run the whole workload in seconds, but causality lets it compute sampled
outputs of the full run exactly: the first samples of a data set's traces, and the gradient
for an adjoint source confined to the first samples.  These comparisons take the longest of
the GPU suite (tens of seconds of FP64 oracle work), so they are collected last.
"""
import numpy as np
import pytest

import pat_synth as ps
from tests._problems import grid_params, oracle_grid, gpu_plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
