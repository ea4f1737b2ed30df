"""GPU forward operator (pat_forward) against the FP64 oracle.

Tolerance: relative L2 error of the traces <= 1e-4 (FP32 stepping against
FP64; the observed error is ~1e-6 at Nt = 400).
"""
import numpy as np
import pytest

from tests._problems import grid_params, oracle_grid, gpu_plan, rel_l2, small_case
import pat_synth as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _oracle_traces(gp, c, p0, xy):
    from oracle.forward import forward
    from oracle.sensors import sensor_matrix
    g = oracle_grid(gp)
    return forward(g, c, p0, sensor_matrix(g, xy))


def test_forward_plain64_matches_oracle():
    w = ps.workload("plain64", 0)
    gp = grid_params(64, 400)
    assert gp["n"] + 2 * gp["pml"] == 108
    ref = _oracle_traces(gp, w.c_true, w.p0_true, w.sensors)
    plan = gpu_plan(gp, w.sensors, 1)
    y = plan.forward(_dev(w.c_true), _dev(w.p0_true)).cpu().numpy()
    assert rel_l2(y, ref) <= 1e-4
    # every time sample individually, relative to the trace amplitude
    assert np.abs(y - ref).max() <= 1e-4 * np.abs(ref).max()


def test_forward_ragged_multi_k_matches_oracle():
    c, p0, xy = small_case()
    gp = grid_params(40, 150)                 # Ng = 80, 41 spectral columns
    ref = _oracle_traces(gp, c, p0, xy)
    plan = gpu_plan(gp, xy, 3)
    y = plan.forward(_dev(c), _dev(p0)).cpu().numpy()
    for k in range(3):
        assert rel_l2(y[k], ref[k]) <= 1e-4


@pytest.mark.parametrize("n,pml", [(16, 8), (12, 12), (20, 20), (100, 22), (50, 20), (8, 10)])
def test_forward_other_grid_sizes(n, pml):
    # Ng = 32 (radix 4,4,2), 36, 60, 144, 90 (= 2 mod 4); Ng = 28 has the factor 7 and is rejected
    from paper_2505_08482_gb300 import _binding as B
    from oracle.grid import is_smooth
    ng = n + 2 * pml
    rng = ps.rng_for(n)
    c = 1450.0 + 100.0 * rng.uniform(size=(n, n))
    p0 = rng.uniform(size=(2, n, n))
    xy = ps.circle_sensors(n, 6, 1e-4, radius_cells=0.3 * n)
    gp = grid_params(n, 40, pml=pml)
    if not is_smooth(ng):
        with pytest.raises(B.PatError):
            gpu_plan(gp, xy, 2)
        return
    ref = _oracle_traces(gp, c, p0, xy)
    y = gpu_plan(gp, xy, 2).forward(_dev(c), _dev(p0)).cpu().numpy()
    assert rel_l2(y, ref) <= 1e-4


def test_forward_single_sample_is_sensor_interpolation():
    c, p0, xy = small_case(K=2)
    gp = grid_params(40, 1)
    ref = _oracle_traces(gp, c, p0, xy)
    y = gpu_plan(gp, xy, 2).forward(_dev(c), _dev(p0)).cpu().numpy()
    assert np.abs(y - ref).max() <= 1e-6 * np.abs(ref).max()


def test_forward_is_linear_in_p0_and_deterministic():
    c, p0, xy = small_case(K=2)
    gp = grid_params(40, 120)
    plan = gpu_plan(gp, xy, 2)
    y1 = plan.forward(_dev(c), _dev(p0)).cpu().numpy()
    y2 = plan.forward(_dev(c), _dev(p0)).cpu().numpy()
    assert np.array_equal(y1, y2)
    y3 = plan.forward(_dev(c), _dev(2.0 * p0)).cpu().numpy()
    assert rel_l2(y3, 2.0 * y1) <= 1e-6


def test_largest_grid_side():
    """The largest supported FFT grid (Ng = 1024 = 984 + 2 x 20, generic passes) against the
    oracle, forward and gradient; one more cell per side (Ng 1026) is rejected."""
    from oracle.adjoint import adjoint_grad
    from oracle.sensors import sensor_matrix
    from paper_2505_08482_gb300 import _binding as B
    n, K, nt = 984, 1, 16
    rng = ps.rng_for(984)
    c = 1500.0 + 60.0 * rng.uniform(size=(n, n))
    p0 = np.zeros((K, n, n))
    p0[0, 480:504, 480:504] = 1.0
    xy = ps.rng_for(985).uniform(470, 514, size=(24, 2)) * 1e-4
    gp = grid_params(n, nt, pml=20)
    plan = gpu_plan(gp, xy, K, ckpt_every=8)
    assert plan.ng == 1024 and plan.variants == 0
    y = plan.forward(_dev(c), _dev(p0)).cpu().numpy()
    g = oracle_grid(gp)
    S = sensor_matrix(g, xy)
    ref = _oracle_traces(gp, c, p0, xy)
    assert rel_l2(y, ref) <= 1e-4
    ym = ref + 0.01 * np.abs(ref).max() * ps.rng_for(986).standard_normal(ref.shape)
    w = np.array([1.0 / np.abs(ref).max() ** 2])
    J, gp0, gc = plan.adjoint_grad(_dev(np.full((n, n), 1500.0)), _dev(0.5 * p0), _dev(ym), _dev(w))
    Jo, gpo, gco = adjoint_grad(g, np.full((n, n), 1500.0), 0.5 * p0, S, ym, w)
    assert abs(J.item() - Jo) <= 1e-4 * Jo
    assert rel_l2(gp0.cpu().numpy(), gpo) <= 1e-3
    assert rel_l2(gc.cpu().numpy(), gco) <= 1e-3
    with pytest.raises(B.PatError):
        gpu_plan(grid_params(986, nt, pml=20), xy, K)
