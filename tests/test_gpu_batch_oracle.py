"""Batched plans against the FP64 oracle, instance by instance.

A batched plan (pat_plan_create_batched) runs each pass once for several
independent instances that share the grid and the sensors but have their own
speed of sound and their own number of data sets.  Here every instance's
traces, objective and gradients (Sec. 3, Eqs. gradient_p0 and gradient_sos)
are compared with the oracle's forward and discrete adjoint for that instance
alone, at a compiled grid side of the multigrid levels (Ng 108) and at the
benchmark's (Ng 300), with mixed K and kernel variant 0.
"""
import numpy as np
import pytest

import pat_synth as ps
from tests._problems import grid_params, gpu_plan, oracle_grid, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("n,Ks,nt", [(64, (1, 3, 8), 90), (256, (1, 2, 3), 60)])
def test_batched_plan_matches_oracle_per_instance(n, Ks, nt):
    from oracle.adjoint import adjoint_grad
    from oracle.forward import forward
    from oracle.sensors import sensor_matrix
    rng = ps.rng_for(21)
    gp = grid_params(n, nt)
    # sensors spread over the central region where the sources lie, so that every data set's
    # waves reach many of them within the short time series
    xy = ps.rng_for(22).uniform(0.25 * n, 0.75 * n, size=(2 * n, 2)) * 1e-4
    cs = [ps.ellipse_phantom(n, 3 + i, rng) for i in range(len(Ks))]
    p0s = [np.stack([ps.blob_p0(n, 4, rng, sigma_cells=(2.0, 4.0)) for _ in range(K)]) for K in Ks]
    plan = gpu_plan(gp, xy, list(Ks), ckpt_every=16)
    assert plan.ng in (108, 300)
    plan.variant = 0
    y = plan.forward(_dev(np.stack(cs)), _dev(np.concatenate(p0s))).cpu().numpy()
    g = oracle_grid(gp)
    S = sensor_matrix(g, xy)
    # gradient at a point away from the truth: per-instance scaled c and halved p0
    c_eval = [1500.0 + 0.9 * (c - 1500.0) for c in cs]
    p0_eval = [0.5 * p for p in p0s]
    y_meas, wts = [], []
    k0 = 0
    for i, K in enumerate(Ks):
        y_ref = forward(g, cs[i], p0s[i], S)
        assert rel_l2(y[k0:k0 + K], y_ref) <= 1e-4, f"instance {i} traces"
        ym = ps.add_noise(y_ref, ps.rng_for(40 + i))
        y_meas.append(ym)
        wts.append(ps.rng_for(60 + i).uniform(0.5, 2.0, size=K) / np.abs(ym).max() ** 2)
        k0 += K
    J, gp0, gc = plan.adjoint_grad(_dev(np.stack(c_eval)), _dev(np.concatenate(p0_eval)),
                                   _dev(np.concatenate(y_meas)), _dev(np.concatenate(wts)))
    J, gp0, gc = J.cpu().numpy(), gp0.cpu().numpy(), gc.cpu().numpy()
    k0 = 0
    for i, K in enumerate(Ks):
        Jo, gpo, gco = adjoint_grad(g, c_eval[i], p0_eval[i], S, y_meas[i], wts[i])
        assert abs(J[i] - Jo) <= 1e-4 * abs(Jo), f"instance {i} J"
        assert rel_l2(gp0[k0:k0 + K], gpo) <= 1e-3, f"instance {i} dJ/dp0"
        assert rel_l2(gc[i], gco) <= 1e-3, f"instance {i} dJ/dc"
        k0 += K
