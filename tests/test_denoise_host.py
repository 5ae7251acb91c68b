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


def _segment_area(field, k):
    """Open area of segment k at the isocentre plane (no leaf gap or
    transmission): sum over pairs of (leaf opening within the X jaws) x
    (pair width within the Y jaws)."""
    e = field.pair_edges
    x0, x1, y0, y1 = field.jaws[k]
    lv = field.leaves[k]
    wx = np.clip(np.minimum(lv[:, 1], x1) - np.maximum(lv[:, 0], x0), 0, None)
    wy = np.clip(np.minimum(e[1:], y1) - np.maximum(e[:-1], y0), 0, None)
    return float((wx * wy).sum())


def test_aperture_fluence_matches_sampled_source_positions():
    """The projected aperture against the oracle's source sampling: primaries
    are drawn uniformly over the open rectangles, MU-weighted, so pixel
    (ix, iy) of the EPID, with ix = floor((X SID/SAD + W/2) / p), receives a
    fraction (sum of MU open over it) x (pixel area at the isocentre) /
    (sum_k MU_k area_k) of them.  Checked on pixels that no aperture edge
    crosses; a transposed or unmagnified map fails it."""
    from oracle import sample_source
    from paper_2510_24154_b300 import workloads as W
    from paper_2510_24154_b300.denoise_data import aperture_fluence

    fld = W.imrt_field(np.random.default_rng(12), 6, gantry_deg=30.0)
    prob = W.config_water_open(npx=96, npy=80, pitch=0.45)
    prob.field = fld
    F = aperture_fluence(fld, prob.epid)
    assert F.shape == (80, 96)
    # the pixel-area average of the same map, from a 16x finer grid
    fine = W.epid_default(96 * 16, 80 * 16, prob.epid.pitch / 16)
    Fa = aperture_fluence(fld, fine).reshape(80, 16, 96, 16).mean(axis=(1, 3))
    assert np.abs(Fa - F).max() <= 1.0 and (Fa == F).mean() > 0.2
    n = 400_000
    X, Y, _ = sample_source(prob, n, seed=5)
    mag = fld.sid / fld.sad
    p = prob.epid.pitch
    ix = np.floor((X * mag + 0.5 * 96 * p) / p).astype(int)
    iy = np.floor((Y * mag + 0.5 * 80 * p) / p).astype(int)
    ok = (ix >= 0) & (ix < 96) & (iy >= 0) & (iy < 80)
    counts = np.zeros((80, 96))
    np.add.at(counts, (iy[ok], ix[ok]), 1.0)
    total = sum(m * _segment_area(fld, k) for k, m in enumerate(fld.mu))
    expect = n * Fa * (p / mag) ** 2 / total
    sel = expect > 30
    assert sel.sum() > 500
    z = (counts[sel] - expect[sel]) / np.sqrt(expect[sel])
    assert abs(z.mean()) < 5 / np.sqrt(sel.sum()) and 0.85 < z.std() < 1.2, (z.mean(), z.std())
    # nothing lands where every segment is closed (3 x 3 neighbourhoods: the
    # 16x grid misses openings narrower than a sixteenth of a pixel)
    Fp = np.pad(Fa, 1)
    shut = np.ones_like(Fa, dtype=bool)
    for dy in range(3):
        for dx in range(3):
            shut &= Fp[dy:dy + 80, dx:dx + 96] == 0
    assert shut.sum() > 500 and counts[shut].sum() == 0
    # the same comparison with the map mirrored about the image centre fails
    zt = (counts[sel] - n * Fa[::-1, ::-1][sel] * (p / mag) ** 2 / total) / np.sqrt(expect[sel])
    assert zt.std() > 3


def test_aux_planes_normalisation():
    from paper_2510_24154_b300 import workloads as W
    from paper_2510_24154_b300.denoise_data import AUX_PLANES, MU_PRIMARY, aux_planes

    prob = W.config_water_open(npx=64, npy=48, pitch=0.6)
    t = np.linspace(0.0, 30.0, 64 * 48).reshape(48, 64)
    a = aux_planes(prob.field, prob.epid, t)
    assert a.shape == (AUX_PLANES, 48, 64)
    assert a[0].mean() == pytest.approx(1.0) and a[2].mean() == pytest.approx(1.0)
    assert np.allclose(a[1], t / 40.0)
    inside = a[0] > 0
    ratio = a[2][inside] / a[0][inside]
    assert np.allclose(ratio / ratio.max(), np.exp(-MU_PRIMARY * (t[inside] - t[inside].min())))
