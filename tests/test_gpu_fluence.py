"""The source fluence on the EPID grid (mc_get_field_fluence) against the
oracle's source sampling: primaries are drawn over the MLC/jaw source
rectangles (MU weights, leaf and jaw transmission, tongue and groove, leaf
gap; Sec. 2.1.1), so EPID pixel (ix, iy), with ix = floor((X SID/SAD + W/2)
/ p), receives a fraction (pixel average of the density) x (pixel area at
the isocentre) of them.  The pixel average is taken from the same call on a
16x finer EPID grid."""
import numpy as np
import pytest

import oracle
from paper_2510_24154_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_24154_b300.binding import MCError, Simulator  # noqa: E402


def _fluence(prob, epid):
    sim = Simulator(prob.physics)
    try:
        sim.init_geometry(prob.phantom, epid)
        sim.set_field(prob.field)
        F = sim.fluence()
        Fd = torch.empty(F.shape, dtype=torch.float64, device="cuda:0")
        sim.fluence_device(Fd)
        torch.cuda.synchronize()
        # segments add their densities with atomics: equal up to summation order
        assert np.allclose(Fd.cpu().numpy(), F, rtol=1e-12, atol=0)
        with pytest.raises(MCError):
            sim.fluence(field=1)
    finally:
        sim.close()
    return F


@pytest.mark.parametrize("modifiers", [{}, {"tg_width": 0.1, "leaf_gap": 0.06, "leaf_transmission": 0.02,
                                            "jaw_transmission": 0.01}])
def test_fluence_matches_sampled_source_positions(modifiers):
    fld = W.imrt_field(np.random.default_rng(12), 6, gantry_deg=30.0)
    for k, v in modifiers.items():
        setattr(fld, k, v)
    prob = W.config_water_open(npx=96, npy=80, pitch=0.45)
    prob.field = fld
    F = _fluence(prob, prob.epid)
    Fa = _fluence(prob, W.epid_default(96 * 16, 80 * 16, prob.epid.pitch / 16)).reshape(80, 16, 96, 16).mean(
        axis=(1, 3))
    # pixel centres and pixel averages agree away from edges
    assert np.isclose(F, Fa, rtol=1e-9, atol=0).mean() > 0.2 and np.abs(F - Fa).max() <= F.max()
    n = 400_000
    X, Y, _ = oracle.sample_source(prob, n, seed=5)
    mag = fld.sid / fld.sad
    p = prob.epid.pitch
    ix = np.floor((X * mag + 0.5 * 96 * p) / p).astype(int)
    iy = np.floor((Y * mag + 0.5 * 80 * p) / p).astype(int)
    ok = (ix >= 0) & (ix < 96) & (iy >= 0) & (iy < 80)
    counts = np.zeros((80, 96))
    np.add.at(counts, (iy[ok], ix[ok]), 1.0)
    area = (p / mag) ** 2
    # the density integrates to the fraction of rays that hit the grid
    assert Fa.sum() * area == pytest.approx(ok.mean(), abs=4 * np.sqrt(ok.mean() * (1 - ok.mean()) / n) + 1e-3)
    expect = n * Fa * area
    sel = expect > 30
    assert sel.sum() > 500
    z = (counts[sel] - expect[sel]) / np.sqrt(expect[sel])
    assert abs(z.mean()) < 5 / np.sqrt(sel.sum()) and 0.85 < z.std() < 1.2, (z.mean(), z.std())
    if not modifiers:
        # nothing lands where every segment is closed (3 x 3 neighbourhoods:
        # the 16x grid misses openings narrower than a sixteenth of a pixel)
        Fp = np.pad(Fa, 1)
        shut = np.ones_like(Fa, dtype=bool)
        for dy in range(3):
            for dx in range(3):
                shut &= Fp[dy:dy + 80, dx:dx + 96] == 0
        assert shut.sum() > 500 and counts[shut].sum() == 0
    # the map mirrored about the image centre fails the same comparison
    zt = (counts[sel] - n * Fa[::-1, ::-1][sel] * area) / np.sqrt(expect[sel])
    assert zt.std() > 3


def test_fluence_and_region_dose_of_every_field_of_a_batch():
    """In a two-field batch each field's fluence equals that of the field
    set up alone, and the region statistic of field 1 is that of its own
    sub-tallies (the other field's histories do not enter it)."""
    from paper_2510_24154_b300 import calibration as CAL
    ep = W.epid_default(96, 80, 0.45)
    f0 = W.imrt_field(np.random.default_rng(3), 4, gantry_deg=0.0)
    f1 = W.imrt_field(np.random.default_rng(4), 7, gantry_deg=90.0)
    f1.tg_width, f1.leaf_gap = 0.1, 0.06
    prob = W.config_water_open(npx=96, npy=80, pitch=0.45)
    sim = Simulator(prob.physics)
    try:
        sim.init_geometry(prob.phantom, ep)
        sim.set_fields([f0, f1])
        both = [sim.fluence(field=f) for f in range(2)]
        for f, fld in enumerate((f0, f1)):
            sim.set_field(fld)
            assert np.allclose(both[f], sim.fluence(), rtol=1e-12, atol=0)
        sim.set_fields([f0, f1])
        sim.run_batch([20_000, 30_000], 9)
        tally = sim.tally(field=1).astype(np.float64) / 2.56e8
        B = tally.shape[0]
        nb = oracle.batch_counts(30_000, B).astype(float)
        _, thick, rho = ep.layers[ep.sensitive]
        conv = 1.602176634e-13 / (rho * ep.pitch ** 2 * thick * 1e-3)
        ix0, ix1, iy0, iy1 = CAL.central_rect(ep, half_cm=3.0)
        reg = tally[:, iy0:iy1, ix0:ix1].reshape(B, -1)
        want = reg.sum() * conv / (30_000 * reg.shape[1])
        per = reg.sum(axis=1) * conv / (nb * reg.shape[1])
        want_sd = np.sqrt(((per - want) ** 2).sum() / (B * (B - 1)))
        m, sd = sim.region_dose(ix0, ix1, iy0, iy1, field=1)
        assert want > 0 and m == pytest.approx(want, rel=1e-12) and sd == pytest.approx(want_sd, rel=1e-9)
        with pytest.raises(MCError):
            sim.region_dose(ix0, ix1, iy0, iy1, field=2)
    finally:
        sim.close()
