"""Every kernel variant (generic Stockham, fixed-size two-level tiles with the state in
registers or staged in shared memory) against the oracle.

Grid sides 108, 144, 180, 200, 240, 300 (domains 64..256 with the automatic
PML) have compiled two-level FFT passes; each variant must reproduce the
oracle's traces (1e-4 relative L2) and gradients (1e-3).
"""
import numpy as np
import pytest

import pat_synth as ps
from tests._problems import grid_params, oracle_grid, gpu_plan, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIDES = {64: 108, 96: 144, 128: 180, 160: 200, 192: 240, 256: 300}


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _case(n, K, M, nt, seed):
    rng = ps.rng_for(seed)
    c = ps.ellipse_phantom(n, 4, rng)
    p0 = np.stack([ps.vessel_p0(n, rng) for _ in range(K)])
    xy = ps.circle_sensors(n, M, 1e-4, phase=0.1)
    return c, p0, xy


@pytest.mark.parametrize("n", sorted(SIDES))
def test_forward_all_variants(n):
    from oracle.forward import forward
    from oracle.sensors import sensor_matrix
    c, p0, xy = _case(n, 2, 32, 60, n)
    gp = grid_params(n, 60)
    assert gp["n"] + 2 * gp["pml"] == SIDES[n]
    g = oracle_grid(gp)
    ref = forward(g, c, p0, sensor_matrix(g, xy))
    plan = gpu_plan(gp, xy, 2)
    assert plan.variants >= 3 and plan.variant == 0
    outs = {}
    for v in range(-1, plan.variants):
        plan.variant = v
        outs[v] = plan.forward(_dev(c), _dev(p0)).cpu().numpy()
        assert rel_l2(outs[v], ref) <= 1e-4, (v, rel_l2(outs[v], ref))
    for v in range(plan.variants):
        assert rel_l2(outs[v], outs[-1]) <= 1e-5, v


@pytest.mark.parametrize("n", sorted(SIDES))
def test_gradient_all_variants(n):
    from oracle.adjoint import adjoint_grad
    from oracle.forward import forward
    from oracle.sensors import sensor_matrix
    c, p0, xy = _case(n, 2, 24, 50, 10 + n)
    gp = grid_params(n, 50)
    g = oracle_grid(gp)
    S = sensor_matrix(g, xy)
    ym = ps.add_noise(forward(g, c, p0, S), ps.rng_for(n))
    # fixed weights: with 50 steps a data set may not reach the sensors yet, and the
    # peak-to-peak noise weight of an empty trace would make J depend on ~1e-9 samples
    wt = np.array([1.0, 2.0])
    c0 = np.full((n, n), 1520.0)
    J, gp0, gc = adjoint_grad(g, c0, 0.5 * p0, S, ym, wt)
    plan = gpu_plan(gp, xy, 2, ckpt_every=16)
    for v in range(-1, plan.variants):
        plan.variant = v
        Jg, a, b = plan.adjoint_grad(_dev(c0), _dev(0.5 * p0), _dev(ym), _dev(wt))
        assert abs(Jg.item() - J) <= 1e-4 * J, v
        assert rel_l2(a.cpu().numpy(), gp0) <= 1e-3, v
        assert rel_l2(b.cpu().numpy(), gc) <= 1e-3, v


def test_variant_selection_errors():
    from paper_2505_08482_gb300 import _binding as B
    c, p0, xy = _case(40, 1, 8, 10, 1)
    plan = gpu_plan(grid_params(40, 10), xy, 1)      # Ng = 80: generic only
    assert plan.variants == 0 and plan.variant == -1
    with pytest.raises(B.PatError):
        plan.variant = 0
