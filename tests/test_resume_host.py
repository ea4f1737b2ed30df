"""Host side of the resumable reconstruction: the state file is tied to its configuration
and inputs, so a run cannot continue from a file written by a different problem."""
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
