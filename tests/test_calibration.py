"""Host logic of the S(t, s) calibration sweep (Sec. 2.2, Eq. 2): slab
geometry, the central 1 cm x 1 cm region, the region statistics and
k = M / S."""
import numpy as np
import pytest

from paper_2510_24154_b300 import calibration as CAL
from paper_2510_24154_b300 import workloads as W


def test_slab_and_region():
    ph = CAL.slab_phantom(10.0)
    assert ph.hu.shape == (80, 20, 80) and (ph.hu == 0).all()
    assert ph.origin[1] == pytest.approx(-5.0)
    air = CAL.slab_phantom(0.0)
    assert air.hu.shape[1] == 1 and (air.hu == -1000).all()
    ep = W.epid_default(1024, 768, 0.039)
    m = CAL.central_region(ep)
    assert m.sum() == 26 * 26                       # centres within 0.5 cm: 12.8 pitches each side
    ys, xs = np.nonzero(m)
    assert (xs.min(), xs.max(), ys.min(), ys.max()) == (499, 524, 371, 396)


def test_region_signal_closed_form():
    ep = W.epid_default(64, 48, 0.25)
    m = CAL.central_region(ep)
    B, n = 16, 1600
    tally = np.full((B, 48, 64), 2.0)              # 2 MeV per pixel per batch
    mean, sd = CAL.region_signal(tally, n, ep, m)
    _, thick, rho = ep.layers[ep.sensitive]
    conv = 1.602176634e-13 / (rho * 0.25 * 0.25 * thick * 1e-3)
    assert mean == pytest.approx(2.0 * B * conv / n, rel=1e-12)
    assert sd == pytest.approx(0.0, abs=1e-30)
    tally[3] *= 3.0                                 # one batch three times hotter
    mean, sd = CAL.region_signal(tally, n, ep, m)
    per = np.full(B, 2.0 * conv / (n / B))
    per[3] *= 3.0
    assert mean == pytest.approx(per.mean(), rel=1e-12)
    assert sd == pytest.approx(per.std(ddof=1) / np.sqrt(B), rel=1e-12)


def test_k_table_is_the_ratio():
    S = np.arange(1.0, 21.0).reshape(4, 5)
    M = 2.0 * S
    M[1, 2] = 3.0 * S[1, 2]
    lut = CAL.k_table(M, S)
    assert lut.k.shape == (4, 5) and lut.k[0, 0] == 2.0 and lut.k[1, 2] == 3.0
    assert list(lut.t_nodes) == list(CAL.T_NODES) and list(lut.s_nodes) == list(CAL.S_NODES)
    with pytest.raises(ValueError):
        CAL.k_table(M[:3], S[:3])
