"""Simple-phantom inputs of Sec. 4.1.1: sensor geometry and value ranges."""
import numpy as np

import pat_synth as ps


def test_square_sensors_follow_the_target_boundary():
    xy = ps.square_sensors()
    assert xy.shape == (236, 2)
    ctr = ps.SIMPLE_MARGIN + ps.SIMPLE_TARGET / 2
    cheb = np.max(np.abs(xy - ctr), axis=1)            # distance to the centre in the max norm
    np.testing.assert_allclose(cheb, ps.SIMPLE_TARGET / 2 + 0.2e-3, rtol=0, atol=1e-12)
    perim = 4 * (ps.SIMPLE_TARGET + 0.4e-3)
    arc = np.sort(np.mod(np.arctan2(xy[:, 1] - ctr, xy[:, 0] - ctr), 2 * np.pi))
    assert np.all(np.diff(arc) > 0)                    # distinct, ordered around the square
    assert np.all((xy > 0) & (xy < ps.SIMPLE_L))       # inside the computational domain
    assert perim / 236 > 0.34e-3


def test_simple_phantom_values():
    for kind, hi, extra in (("circles", 1580.0, None), ("water", 1580.0, 1482.0), ("bone", 2500.0, 2500.0)):
        c = ps.simple_phantom_c(kind, 136)
        assert c.min() == 1430.0 and c.max() == hi
        if extra is not None:
            assert np.any(np.isclose(c, extra))
    p0 = ps.simple_phantom_p0(136, K=4)
    assert p0.shape == (4, 136, 136) and p0.min() == 0.0 and p0.max() == 10.0
    assert not np.allclose(p0[0], p0[1])
