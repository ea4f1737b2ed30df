"""Host side of the resumable reconstruction: the state file is tied to its configuration,
inputs and targets, so a run cannot continue from a file written by a different problem; and the
level-by-level bookkeeping (which levels run again, report rows, status, the finished file) is
checked with CPU stand-ins for the device calls."""
import pytest

torch = pytest.importorskip("torch")


def test_resume_fingerprint_tracks_config_and_inputs():
    import dataclasses
    import numpy as np
    import torch
    from paper_2505_08482_gb300.solver import ReconConfig, _fingerprint
    xy = np.zeros((4, 2))
    cfg = ReconConfig(levels=(32, 64), L=6.4e-3, dt_data=1e-8, nt_data=10, sensors_xy=xy, K=1)
    a, b = torch.zeros(3), torch.ones(2, 2)
    f = _fingerprint(cfg, (a, b))
    assert f == _fingerprint(cfg, (a.clone(), b.clone()))
    assert f != _fingerprint(dataclasses.replace(cfg, iters=7), (a, b))
    assert f != _fingerprint(dataclasses.replace(cfg, levels=(64,)), (a, b))
    assert f != _fingerprint(cfg, (a, b * 2))
    assert f != _fingerprint(dataclasses.replace(cfg, sensors_xy=xy + 1e-3), (a, b))


def test_resume_fingerprint_tracks_targets():
    import numpy as np
    from paper_2505_08482_gb300.solver import ReconConfig, _fingerprint
    cfg = ReconConfig(levels=(32, 64), L=6.4e-3, dt_data=1e-8, nt_data=10, sensors_xy=np.zeros((4, 2)), K=1)
    a = torch.zeros(3)
    f = _fingerprint(cfg, (a,), extra=[[2.0, 0.0, True, False]])
    assert f == _fingerprint(cfg, (a,), extra=[[2.0, 0.0, True, False]])
    assert f != _fingerprint(cfg, (a,), extra=[[2.5, 0.0, True, False]])
    assert f != _fingerprint(cfg, (a,), extra=[[2.0, 0.0, False, False]])


def _fake_library(monkeypatch, calls):
    """CPU stand-ins for the device calls of the resumable driver: prolongation by nearest cell and
    a 'reconstruction' that adds one to every field and reports one row per instance, so that the
    state file's bookkeeping is checked without a GPU."""
    import numpy as np
    from paper_2505_08482_gb300 import solver

    def prolong(src, n_dst, stream=None):
        n = src.shape[-1]
        idx = torch.as_tensor((np.arange(n_dst) * n) // n_dst)
        return src[:, idx][:, :, idx].contiguous()

    def reconstruct_batched(cfg, instances, stream=None, max_report=4096):
        calls.append(int(cfg.levels[0]))
        out = []
        for i, ins in enumerate(instances):
            n = int(cfg.levels[0])
            assert tuple(ins["c_init"].shape) == (n, n)
            status = -6 if (i == 1 and n == 32) else 0   # a failed line search on one level
            out.append((ins["c_init"] + 1.0, ins["p0_init"] + 1.0,
                        [dict(level=0, it=0, J=float(n), gnorm=1.0, alpha=1.0, trials=1, J_new=0.5 * n, ms=1.0,
                              Ec=-1.0, Ep0=-1.0)], status))
        return out, 2.0

    monkeypatch.setattr(solver, "_f32", lambda t, shape, name, device: t)
    monkeypatch.setattr(solver, "prolong", prolong)
    monkeypatch.setattr(solver, "reconstruct_batched", reconstruct_batched)
    return solver


def _instances(n=64):
    return [dict(y_meas=torch.zeros(1, 5, 4), w=torch.ones(1), c_init=torch.full((n, n), 1500.0)),
            dict(y_meas=torch.ones(2, 5, 4), w=torch.ones(2), c_init=torch.full((n, n), 1400.0),
                 p0_init=torch.zeros(2, n, n))]


def test_resumable_driver_bookkeeping(monkeypatch, tmp_path):
    import numpy as np
    calls = []
    solver = _fake_library(monkeypatch, calls)
    cfg = solver.ReconConfig(levels=(16, 32, 64), L=6.4e-3, dt_data=1e-8, nt_data=5, sensors_xy=np.zeros((4, 2)),
                             K=1)
    whole, total, done = solver.reconstruct_batched_resumable(cfg, _instances(), str(tmp_path / "a.npz"))
    assert done == 3 and calls == [16, 32, 64] and total == 6.0
    calls.clear()
    path = str(tmp_path / "b.npz")
    part, _, done = solver.reconstruct_batched_resumable(cfg, _instances(), path, stop_after_level=1)
    assert done == 2 and calls == [16, 32] and tuple(part[0][0].shape) == (32, 32)
    calls.clear()
    res, total, done = solver.reconstruct_batched_resumable(cfg, _instances(), path)
    assert done == 3 and calls == [64] and total == 6.0   # only the last level runs again
    for (c, p0, rows, st), (cw, p0w, rowsw, stw), ins in zip(res, whole, _instances()):
        assert torch.equal(c, cw) and torch.equal(p0, p0w) and rows == rowsw and st == stw
        assert [r["level"] for r in rows] == [0, 1, 2]
        assert float(c[0, 0]) == float(ins["c_init"][0, 0]) + 3.0   # one step per level, each from the last
    assert res[1][3] == -6 and res[0][3] == 0                 # a level's failed search is kept
    calls.clear()
    again, _, done = solver.reconstruct_batched_resumable(cfg, _instances(), path)
    assert done == 3 and calls == []                          # a finished file: nothing runs
    insts = _instances()
    insts[1]["w"] = 2.0 * insts[1]["w"]
    with pytest.raises(ValueError):
        solver.reconstruct_batched_resumable(cfg, insts, path)
