"""Resuming a reconstruction from a host file at a multigrid level boundary.

At a level boundary the method starts a new optimisation from the prolonged point with an
empty L-BFGS memory (Sec. 3.1), so a run stopped after a level and resumed from the saved
iterate must give the result of one uninterrupted pat_reconstruct bit for bit (kernel variant
fixed), with the same per-iteration report.
"""
import numpy as np
import pytest

import pat_synth as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _problem():
    from oracle.forward import forward
    from oracle.grid import make_grid
    from oracle.sensors import sensor_matrix
    from paper_2505_08482_gb300.solver import ReconConfig
    w = ps.workload("plain64", 3)
    g = make_grid(64, w.dx, 300, c_ref=1750.0)
    y = ps.add_noise(forward(g, w.c_true, w.p0_true, sensor_matrix(g, w.sensors)), ps.rng_for(103))
    wt = ps.noise_weights(y)
    c_init = 0.5 * (w.c_true.min() + w.c_true.max())
    cfg = ReconConfig(levels=(32, 48, 64), L=64 * w.dx, dt_data=g.dt, nt_data=g.nt, sensors_xy=w.sensors, K=1,
                      mem=20, iters=3, rtol=0.0, ckpt_every=32, autotune=False)
    return cfg, _dev(y), _dev(wt), _dev(np.full((64, 64), c_init))


KEYS = ("level", "it", "J", "gnorm", "alpha", "trials", "J_new")


def test_resume_after_each_level_is_bit_identical(tmp_path):
    from paper_2505_08482_gb300.solver import reconstruct, reconstruct_resumable
    cfg, y, wt, c0 = _problem()
    c_ref, p0_ref, rows_ref, st_ref, _ = reconstruct(cfg, y, wt, c0)
    path = str(tmp_path / "state.npz")
    c1, p01, rows1, _, _, done1 = reconstruct_resumable(cfg, y, wt, c0, path, stop_after_level=0)
    assert done1 == 1 and tuple(c1.shape) == (32, 32) and tuple(p01.shape) == (1, 32, 32)
    assert all(r["level"] == 0 for r in rows1)
    c2, _, _, _, _, done2 = reconstruct_resumable(cfg, y, wt, c0, path, stop_after_level=1)
    assert done2 == 2 and tuple(c2.shape) == (48, 48)
    c3, p03, rows3, st3, _, done3 = reconstruct_resumable(cfg, y, wt, c0, path)
    assert done3 == 3
    assert torch.equal(c3, c_ref) and torch.equal(p03, p0_ref)
    assert st3 == st_ref
    assert [[r[k] for k in KEYS] for r in rows3] == [[r[k] for k in KEYS] for r in rows_ref]
    # a finished state file: nothing left to run, the same result
    c4, p04, rows4, _, _, done4 = reconstruct_resumable(cfg, y, wt, c0, path)
    assert done4 == 3 and torch.equal(c4, c_ref) and torch.equal(p04, p0_ref) and len(rows4) == len(rows_ref)


def test_uninterrupted_resumable_run_matches_and_other_inputs_are_refused(tmp_path):
    from paper_2505_08482_gb300.solver import reconstruct, reconstruct_resumable
    cfg, y, wt, c0 = _problem()
    c_ref, p0_ref, _, _, _ = reconstruct(cfg, y, wt, c0)
    path = str(tmp_path / "state.npz")
    c, p0, _, _, _, done = reconstruct_resumable(cfg, y, wt, c0, path)
    assert done == 3 and torch.equal(c, c_ref) and torch.equal(p0, p0_ref)
    with pytest.raises(ValueError):
        reconstruct_resumable(cfg, y, 2.0 * wt, c0, path)


def _instance(seed, with_truth=False, with_p0=False):
    from oracle.forward import forward
    from oracle.grid import make_grid
    from oracle.sensors import sensor_matrix
    w = ps.workload("plain64", seed)
    g = make_grid(64, w.dx, 300, c_ref=1750.0)
    y = ps.add_noise(forward(g, w.c_true, w.p0_true, sensor_matrix(g, w.sensors)), ps.rng_for(100 + seed))
    ins = {"y_meas": _dev(y), "w": _dev(ps.noise_weights(y)),
           "c_init": _dev(np.full((64, 64), 0.5 * (w.c_true.min() + w.c_true.max())))}
    if with_truth:
        ins.update(c_true=_dev(w.c_true), p0_true=_dev(w.p0_true), ec_target=2.5)
    if with_p0:
        ins["p0_init"] = _dev(0.25 * w.p0_true)
    return ins


def test_batched_resume_is_bit_identical(tmp_path):
    from paper_2505_08482_gb300.solver import reconstruct_batched, reconstruct_batched_resumable
    cfg, _, _, _ = _problem()
    instances = [_instance(3), _instance(4, with_truth=True), _instance(5, with_p0=True)]
    ref, _ = reconstruct_batched(cfg, instances)
    path = str(tmp_path / "batch.npz")
    part, _, done = reconstruct_batched_resumable(cfg, instances, path, stop_after_level=0)
    assert done == 1 and all(tuple(c.shape) == (32, 32) for c, _, _, _ in part)
    res, _, done = reconstruct_batched_resumable(cfg, instances, path)
    assert done == 3
    keys = KEYS + ("Ec", "Ep0")
    for (c, p0, rows, st), (cr, p0r, rowsr, str_) in zip(res, ref):
        assert torch.equal(c, cr) and torch.equal(p0, p0r) and st == str_
        assert [[r[k] for k in keys] for r in rows] == [[r[k] for k in keys] for r in rowsr]
    with pytest.raises(ValueError):
        reconstruct_batched_resumable(cfg, instances[:2], path)
