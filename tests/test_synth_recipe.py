"""The synthetic input recipe (stand-ins for the paper's phantoms and data).

Checks the properties the workloads are stated to have: c inclusions in
[1400, 1650] m/s on a 1500 m/s background (cf. 1430 / 1580 m/s of Sec. 4.1.1),
non-negative initial pressures (vessel maps clipped at 1), circle sensors at
0.4375 N cells from the centre and inside the domain, 1 % Gaussian noise of
each data set's peak-to-peak (Sec. 4.1.1), weights from the noisy
peak-to-peak (Sec. 4.1.2), and the same arrays for the same seed.
"""
import numpy as np
import pytest

import pat_synth as ps


@pytest.mark.parametrize("name,n,K,M,nt", [("plain64", 64, 1, 64, 400), ("vessels128", 128, 4, 256, 900),
                                          ("tiny16", 16, 2, 12, 60)])
def test_workload_shapes_ranges_and_determinism(name, n, K, M, nt):
    w = ps.workload(name, 3)
    assert (w.n, w.k, w.m, w.nt, w.dx) == (n, K, M, nt, 1e-4)
    assert w.c_true.shape == (n, n) and w.p0_true.shape == (K, n, n)
    vals = np.unique(w.c_true)
    assert np.all((vals == 1500.0) | ((vals >= 1400.0) & (vals <= 1650.0)))
    assert np.sum(w.c_true != 1500.0) > 0
    assert w.p0_true.min() >= 0.0 and w.p0_true.max() > 0.1
    if name.startswith("vessels"):
        assert w.p0_true.max() <= 1.0
    r = np.hypot(w.sensors[:, 0] - n * w.dx / 2, w.sensors[:, 1] - n * w.dx / 2)
    np.testing.assert_allclose(r, 0.4375 * n * w.dx, rtol=1e-12)
    assert np.all((w.sensors > 0) & (w.sensors < n * w.dx))
    w2 = ps.workload(name, 3)
    assert np.array_equal(w.c_true, w2.c_true) and np.array_equal(w.p0_true, w2.p0_true)
    assert not np.array_equal(w.p0_true, ps.workload(name, 4).p0_true)


def test_noise_is_one_percent_of_each_data_sets_peak_to_peak():
    y = np.stack([np.sin(np.linspace(0, 40, 20000)).reshape(1000, 20) * a for a in (1.0, 5.0, 0.2)])
    yn = ps.add_noise(y, ps.rng_for(1))
    for k, a in enumerate((1.0, 5.0, 0.2)):
        p2p = y[k].max() - y[k].min()
        assert np.std(yn[k] - y[k]) == pytest.approx(0.01 * p2p, rel=0.03)
        assert abs(np.mean(yn[k] - y[k])) < 0.01 * p2p * 0.05
    w = ps.noise_weights(yn)
    for k in range(3):
        assert w[k] == pytest.approx(1.0 / (0.01 * (yn[k].max() - yn[k].min())) ** 2, rel=1e-12)
    assert np.array_equal(yn, ps.add_noise(y, ps.rng_for(1)))


def test_blob_and_vessel_maps():
    rng = ps.rng_for(9)
    b = ps.blob_p0(64, 5, rng)
    assert b.min() >= 0.0 and 0.5 <= b.max() <= 5.0
    v = ps.vessel_p0(64, rng)
    assert v.min() >= 0.0 and v.max() <= 1.0 and np.mean(v > 0.05) < 0.5
