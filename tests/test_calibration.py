"""Host logic of the S(t, s) calibration sweep (Sec. 2.2, Eq. 2): slab
geometry, the central 1 cm x 1 cm region and k = M / S (the region
statistics are the library's, checked on the GPU)."""
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


def test_central_rect_is_the_mask():
    for ep in (W.epid_default(1024, 768, 0.039), W.epid_default(64, 48, 0.25), W.epid_default(65, 47, 0.3)):
        ix0, ix1, iy0, iy1 = CAL.central_rect(ep)
        xs = ((np.arange(ep.npx) + 0.5) - ep.npx / 2) * ep.pitch
        ys = ((np.arange(ep.npy) + 0.5) - ep.npy / 2) * ep.pitch
        assert list(np.nonzero(np.abs(xs) <= 0.5)[0]) == list(range(ix0, ix1))
        assert list(np.nonzero(np.abs(ys) <= 0.5)[0]) == list(range(iy0, iy1))
    with pytest.raises(ValueError):
        CAL.central_rect(W.epid_default(2, 2, 2.0))               # pixel centres 1 cm from the centre


def test_k_table_is_the_ratio():
    S = np.arange(1.0, 21.0).reshape(4, 5)
    M = 2.0 * S
    M[1, 2] = 3.0 * S[1, 2]
    lut = CAL.k_table(M, S)
    assert lut.k.shape == (4, 5) and lut.k[0, 0] == 2.0 and lut.k[1, 2] == 3.0
    assert list(lut.t_nodes) == list(CAL.T_NODES) and list(lut.s_nodes) == list(CAL.S_NODES)
    with pytest.raises(ValueError):
        CAL.k_table(M[:3], S[:3])
