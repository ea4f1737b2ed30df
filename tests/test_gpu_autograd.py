"""autograd.Function over (p0, c): oracle gradient and central finite differences."""
import numpy as np
import pytest

import pat_synth as ps
from tests._problems import grid_params, oracle_grid, gpu_plan, rel_l2, small_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def test_autograd_matches_oracle_gradient():
    from oracle.adjoint import adjoint_grad
    from oracle.forward import forward
    from oracle.sensors import sensor_matrix
    from paper_2505_08482_gb300.autograd import data_misfit, pat_forward
    c, p0, xy = small_case(K=2, nt=120)
    gp = grid_params(40, 120)
    g = oracle_grid(gp)
    S = sensor_matrix(g, xy)
    ym = ps.add_noise(forward(g, c, p0, S), ps.rng_for(8))
    wt = ps.noise_weights(ym)
    c0 = np.full((40, 40), 1505.0)
    J, gp0, gc = adjoint_grad(g, c0, 0.5 * p0, S, ym, wt)
    plan = gpu_plan(gp, xy, 2, ckpt_every=16)
    p0t = _dev(0.5 * p0).requires_grad_(True)
    ct = _dev(c0).requires_grad_(True)
    L = data_misfit(pat_forward(p0t, ct, plan), _dev(ym), _dev(wt))
    L.backward()
    assert abs(L.item() - J) <= 1e-4 * J
    assert rel_l2(p0t.grad.cpu().numpy(), gp0) <= 1e-3
    assert rel_l2(ct.grad.cpu().numpy(), gc) <= 1e-3


@pytest.mark.parametrize("name,n,ndir", [("vessels128", 128, 4), ("vessels256", 256, 16)])
def test_autograd_central_differences(name, n, ndir):
    # h = 1e-3 relative; FP32 forward, FP64 misfit: tolerance 2e-2 on each directional derivative
    from paper_2505_08482_gb300.autograd import data_misfit, pat_forward
    w = ps.workload(name, 0)
    gp = grid_params(n, w.nt)
    plan = gpu_plan(gp, w.sensors, w.k, ckpt_every=32)
    y = plan.forward(_dev(w.c_true), _dev(w.p0_true))
    ym = _dev(ps.add_noise(y.cpu().numpy(), ps.rng_for(3)))
    wt = _dev(ps.noise_weights(ym.cpu().numpy()))
    c_init = 0.5 * (w.c_true.min() + w.c_true.max())
    p0t = _dev(0.6 * w.p0_true).requires_grad_(True)
    ct = _dev(np.full((n, n), c_init)).requires_grad_(True)
    L = data_misfit(pat_forward(p0t, ct, plan), ym, wt)
    L.backward()
    gp0, gc = p0t.grad.double(), ct.grad.double()
    rng = ps.rng_for(77)
    for _ in range(ndir):
        dp = torch.as_tensor(rng.standard_normal(p0t.shape), device="cuda")
        dc = torch.as_tensor(rng.standard_normal(ct.shape), device="cuda")
        hp = 1e-3 * float(p0t.detach().abs().max())
        hc = 1e-3 * c_init
        with torch.no_grad():
            Jp = data_misfit(plan.forward((ct.double() + hc * dc).float(), (p0t.double() + hp * dp).float()), ym, wt)
            Jm = data_misfit(plan.forward((ct.double() - hc * dc).float(), (p0t.double() - hp * dp).float()), ym, wt)
        fd = float(Jp - Jm) / 2.0
        an = float(hp * (gp0 * dp).sum() + hc * (gc * dc).sum())
        assert abs(fd - an) <= 2e-2 * abs(an), (fd, an)
