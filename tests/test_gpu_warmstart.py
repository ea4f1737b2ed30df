"""Learned warm start pipeline: solver-generated pairs, training, E_c-tracked reconstruction,
and the gain over the plain start on held-out seeds."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_pairs_training_and_tracked_reconstruction():
    from paper_2505_08482_gb300.solver import ReconConfig, reconstruct_batched
    from paper_2505_08482_gb300.warmstart import (PairGenerator, UNet, init_params, predict_c, relative_error,
                                                  train)
    gen = PairGenerator(n=64, K=2, M=64, nt=300, batch=16)
    X, T, raw = gen.make(list(range(48)), keep_data=True)
    assert X.shape == (48, 2, 64, 64) and T.shape == (48, 64, 64)
    assert torch.isfinite(X).all() and torch.allclose(X.abs().amax(dim=(1, 2, 3)), torch.ones(48, device="cuda"))
    c_true = torch.stack([r["c_true"] for r in raw])
    assert torch.allclose(T, (c_true - 1500.0) / 100.0)
    # the back-projection is the adjoint at constant c0: linear in the data
    net = UNet(3, 16, 2, 64, 64, max_batch=16)
    net.set_params(init_params(3, 16, 2, seed=0))
    hist = train(net, X, T, epochs=15, batch=16, lr=2e-3)
    assert hist[-1] < hist[0]
    c_pred = predict_c(net, X)
    c_const = torch.full_like(c_true, 1500.0)
    e_pred = relative_error(c_pred, c_true).mean().item()
    e_const = relative_error(c_const, c_true).mean().item()
    print(f"training-set E_c: network {e_pred:.2f} % vs constant 1500 m/s {e_const:.2f} %")
    assert e_pred < e_const
    cfg = ReconConfig(levels=(32, 64), L=64e-4, dt_data=gen.gs.dt, nt_data=gen.nt, sensors_xy=gen.sensors, K=2,
                      iters=3, mem=5, ckpt_every=32, rtol=0.0)
    insts = [dict(y_meas=r["y_meas"].contiguous(), w=r["w"].contiguous(), c_init=c_pred[j].contiguous(),
                  c_true=r["c_true"].contiguous(), ec_target=0.01) for j, r in enumerate(raw[:4])]
    res, ms = reconstruct_batched(cfg, insts)
    for j, (c, p0, rows, st) in enumerate(res):
        assert len(rows) == 6 and all(r["Ec"] >= 0 for r in rows)
        # the tracked E_c of the last finest-level iteration is the error of the returned c
        assert abs(rows[-1]["Ec"] - relative_error(c[None], c_true[j][None]).item()) < 1e-3


def test_warm_start_gain_on_held_out_seeds():
    """What the network gains over the paper's plain start (c = midpoint of the true range,
    Sec. 4.1.2) on seeds it never saw: a lower initial E_c, at least as many instances reaching
    the E_c target and fewer L-BFGS iterations to reach it (unreached counted as the budget + 1)."""
    import numpy as np
    from paper_2505_08482_gb300.solver import ReconConfig, reconstruct_batched
    from paper_2505_08482_gb300.warmstart import (PairGenerator, UNet, init_params, iterations_to, predict_c,
                                                  relative_error, train)
    gen = PairGenerator(n=64, K=2, M=64, nt=300, batch=64)
    X, T, _ = gen.make(list(range(2048)))
    net = UNet(3, 16, 2, 64, 64, max_batch=32)
    net.set_params(init_params(3, 16, 2, seed=3))
    hist = train(net, X, T, epochs=20, batch=32, lr=2e-3)
    assert hist[-1] < hist[0]
    del X, T
    Xh, _, raw = gen.make(list(range(10 ** 6, 10 ** 6 + 32)), keep_data=True)
    c_true = torch.stack([r["c_true"] for r in raw])
    c_warm = predict_c(net, Xh)
    c_plain = torch.stack([torch.full_like(ct, 0.5 * float(ct.min() + ct.max())) for ct in c_true])
    e_warm0 = relative_error(c_warm, c_true).cpu().numpy()
    e_plain0 = relative_error(c_plain, c_true).cpu().numpy()
    target, iters = 2.0, 10
    cfg = ReconConfig(levels=(32, 64), L=64e-4, dt_data=gen.gs.dt, nt_data=gen.nt, sensors_xy=gen.sensors, K=2,
                      iters=iters, mem=20, ckpt_every=32, rtol=0.0)
    out = {}
    for name, cinit in (("plain", c_plain), ("warm", c_warm)):
        insts = [dict(y_meas=r["y_meas"].contiguous(), w=r["w"].contiguous(), c_init=cinit[j].contiguous(),
                      c_true=r["c_true"].contiguous(), ec_target=target) for j, r in enumerate(raw)]
        res, _ = reconstruct_batched(cfg, insts)
        its = [iterations_to(rows, target, 2)[0] for _, _, rows, _ in res]
        out[name] = (sum(i is not None for i in its) / len(its),
                     float(np.mean([i if i is not None else 2 * iters + 1 for i in its])))
    print(f"held-out initial E_c median: warm {np.median(e_warm0):.2f} % vs plain {np.median(e_plain0):.2f} %; "
          f"reached {target} %: warm {out['warm'][0]:.2f} vs plain {out['plain'][0]:.2f}; "
          f"mean iterations: warm {out['warm'][1]:.2f} vs plain {out['plain'][1]:.2f}")
    assert np.median(e_warm0) < np.median(e_plain0)
    assert out["warm"][0] >= out["plain"][0]
    assert out["warm"][1] < out["plain"][1]
