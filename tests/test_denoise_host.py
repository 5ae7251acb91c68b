"""Host logic of the denoiser experiment (no GPU): the plain-Monte-Carlo
history count that matches a quality target, interpolated in log N."""
import numpy as np
import pytest

pytest.importorskip("torch")
from paper_2510_24154_b300.denoise_data import bin_image, matched_histories  # noqa: E402


def test_matched_histories_log_interpolation():
    ladder = [(1e7, 0.5), (1e8, 0.7), (1e9, 0.9)]
    assert matched_histories(ladder, 0.7) == pytest.approx(1e8)
    # halfway between 0.7 and 0.9 in value is halfway in log N
    assert matched_histories(ladder, 0.8) == pytest.approx(np.sqrt(1e8 * 1e9))
    assert matched_histories(ladder, 0.4) == 1e7            # already reached at the first count
    assert matched_histories(ladder, 0.95) is None          # never reached
    assert matched_histories(list(reversed(ladder)), 0.6) == pytest.approx(np.sqrt(1e7 * 1e8))


def test_matched_histories_falling_measure():
    # an error that falls with N is matched through its negation
    rms = [(1e7, 0.3), (1e8, 0.1), (1e9, 0.03)]
    n = matched_histories([(k, -v) for k, v in rms], -0.1)
    assert n == pytest.approx(1e8)


def test_bin_image_sums_blocks():
    img = np.arange(24, dtype=float).reshape(4, 6)
    out = bin_image(img, 2)
    assert out.shape == (2, 3)
    assert out[0, 0] == pytest.approx((0 + 1 + 6 + 7) / 4)           # block means
    assert bin_image(np.ones((5, 7)), 2).shape == (2, 3)             # ragged edges dropped


def test_aux_planes_normalisation():
    import torch
    from paper_2510_24154_b300.denoise_data import AUX_PLANES, MU_PRIMARY, aux_planes

    r = np.random.default_rng(2)
    F = torch.tensor(np.where(r.random((48, 64)) < 0.4, 0.0, r.uniform(0.5, 2.0, (48, 64))))
    t = torch.tensor(np.linspace(0.0, 30.0, 64 * 48).reshape(48, 64))
    a = aux_planes(F, t).numpy()
    assert a.shape == (AUX_PLANES, 48, 64)
    assert a[0].mean() == pytest.approx(1.0) and a[2].mean() == pytest.approx(1.0)
    assert np.allclose(a[0] / a[0].max(), F.numpy() / F.numpy().max())
    assert np.allclose(a[1], t.numpy() / 40.0)
    inside = a[0] > 0
    ratio = a[2][inside] / a[0][inside]
    tt = t.numpy()[inside]
    assert np.allclose(ratio / ratio.max(), np.exp(-MU_PRIMARY * (tt - tt.min())))
    assert (a[2][~inside] == 0).all()
