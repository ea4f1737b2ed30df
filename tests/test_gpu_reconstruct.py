"""GPU reconstruction (pat_reconstruct) against the oracle's projected L-BFGS / multigrid.

The reconstruction is non-unique and its late iterations are chaotic, so the
parity is iteration-level: J and ||g|| of the first iterations agree to 1e-3
and the same step lengths are accepted; afterwards only the monotone decrease
of J, the bounds and the improvement of the errors are checked.
"""
import numpy as np
import pytest

import pat_synth as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _data(n, nt, seed, name="plain64"):
    from oracle.forward import forward
    from oracle.grid import make_grid
    from oracle.sensors import sensor_matrix
    w = ps.workload(name, seed)
    g = make_grid(n, w.dx, nt, c_ref=1750.0)
    y = forward(g, w.c_true, w.p0_true, sensor_matrix(g, w.sensors))
    y = ps.add_noise(y, ps.rng_for(100 + seed))
    return w, g, y, ps.noise_weights(y)


@pytest.mark.parametrize("mem,levels", [(20, (64,)), (0, (64,)), (20, (32, 64))])
def test_first_iterations_match_oracle(mem, levels):
    from oracle.multigrid import reconstruct as oracle_recon
    from paper_2505_08482_gb300.solver import ReconConfig, reconstruct
    w, g, y, wt = _data(64, 300, 0)
    c_init = 0.5 * (w.c_true.min() + w.c_true.max())
    T = (g.nt - 1) * g.dt
    iters = 3
    p0_o, c_o, hist = oracle_recon(list(levels), 64 * w.dx, T, w.sensors, y, g.dt, wt, c_init, (1350.0, 1750.0),
                                   iters=iters, mem=mem, rtol=0.0)
    cfg = ReconConfig(levels=levels, L=64 * w.dx, dt_data=g.dt, nt_data=g.nt, sensors_xy=w.sensors, K=1,
                      mem=mem, iters=iters, rtol=0.0, ckpt_every=32)
    c_g, p0_g, rows, status, ms = reconstruct(cfg, _dev(y), _dev(wt), _dev(np.full((64, 64), c_init)))
    ref = [(h["level"], e) for h in hist for e in h["result"].history]
    assert len(rows) == len(ref)
    for r, (lv, e) in zip(rows, ref):
        assert r["level"] == lv and r["it"] == e["it"]
        assert abs(r["J"] - e["J"]) <= 1e-3 * e["J"]
        assert abs(r["gnorm"] - e["gnorm"]) <= 1e-3 * e["gnorm"]
        assert r["alpha"] == e["alpha"]
        assert r["trials"] == e["trials"]


def test_reconstruction_improves_and_respects_bounds():
    from oracle.metrics import relative_error
    from paper_2505_08482_gb300.solver import ReconConfig, reconstruct
    w, g, y, wt = _data(64, 400, 1)
    c_init = 0.5 * (w.c_true.min() + w.c_true.max())
    cfg = ReconConfig(levels=(32, 64), L=64 * w.dx, dt_data=g.dt, nt_data=g.nt, sensors_xy=w.sensors, K=1,
                      iters=10, mem=20)
    c_g, p0_g, rows, status, ms = reconstruct(cfg, _dev(y), _dev(wt), _dev(np.full((64, 64), c_init)))
    c_g, p0_g = c_g.cpu().numpy(), p0_g.cpu().numpy()
    for lv in (0, 1):
        Js = [r["J_new"] for r in rows if r["level"] == lv]
        assert all(b <= a for a, b in zip(Js, Js[1:]))
    assert p0_g.min() >= 0.0 and c_g.min() >= 1350.0 and c_g.max() <= 1750.0
    assert relative_error(w.p0_true, p0_g) < 60.0
    assert relative_error(w.c_true, c_g) <= relative_error(w.c_true, np.full_like(c_g, c_init))
