"""GPU S(t, s) sweep: the trends of beam attenuation and phantom scatter, and
parity of one calibration point with the FP64 oracle (same histories)."""
import numpy as np
import pytest

import oracle
from paper_2510_24154_b300 import calibration as CAL
from paper_2510_24154_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def test_region_dose_is_the_tally_statistic():
    """mc_get_region_dose against the same statistic taken from the raw
    sub-tallies: mean = sum of the region's deposits / (N pixels), error =
    the batch standard error of the per-batch region means; and its
    argument checks."""
    from paper_2510_24154_b300.binding import MCError, Simulator
    ep = W.epid_default(128, 96, 0.312)
    sim = Simulator(W.Physics(coupled=True))
    try:
        sim.init_geometry(CAL.slab_phantom(5.0), ep)
        sim.set_field(W.open_field(8.0, 8.0))
        n = 300_001                                  # B does not divide it
        sim.run(n, 7)
        tally = sim.tally().astype(np.float64) / 2.56e8
        B = tally.shape[0]
        nb = oracle.batch_counts(n, B).astype(float)
        _, thick, rho = ep.layers[ep.sensitive]
        conv = 1.602176634e-13 / (rho * ep.pitch ** 2 * thick * 1e-3)
        for rect in (CAL.central_rect(ep), (0, 128, 0, 96), (5, 6, 90, 96), (60, 70, 40, 41)):
            ix0, ix1, iy0, iy1 = rect
            reg = tally[:, iy0:iy1, ix0:ix1].reshape(B, -1)
            want = reg.sum() * conv / (n * reg.shape[1])
            per = reg.sum(axis=1) * conv / (nb * reg.shape[1])
            want_sd = np.sqrt(((per - want) ** 2).sum() / (B * (B - 1)))
            m, sd = sim.region_dose(*rect)
            assert m == pytest.approx(want, rel=1e-12, abs=1e-300) and sd == pytest.approx(want_sd, rel=1e-9, abs=1e-300)
        for bad in ((0, 0, 0, 1), (-1, 3, 0, 1), (0, 129, 0, 1), (0, 1, 5, 4)):
            with pytest.raises(MCError):
                sim.region_dose(*bad)
    finally:
        sim.close()


def test_s_table_trends():
    ep = W.epid_default(256, 192, 0.156)
    S, U = CAL.s_table(1e6, epid=ep)
    assert S.shape == (4, 5) and (S > 0).all() and (U > 0).all()
    assert (U / S < 0.035).all()          # about 1.5-2.5 %; the batch estimate itself varies ~20 %
    # attenuation: S falls with thickness for every field size
    assert (np.diff(S, axis=1) < 0).all()
    # phantom scatter: behind 10-20 cm, larger fields give more central signal
    assert (np.diff(S[:, 2:], axis=0) > -3 * np.hypot(U[1:, 2:], U[:-1, 2:])).all()
    assert S[3, 4] > S[0, 4]
    # effective attenuation of a 6 MV beam through 20 cm of water (small field)
    mu_eff = -np.log(S[0, 4] / S[0, 0]) / 20.0
    assert 0.03 < mu_eff < 0.06


def test_calibration_point_matches_oracle():
    ep = W.epid_default(128, 96, 0.312)
    t, s, n = 10.0, 10.0, 400_000
    mask = CAL.central_region(ep)
    S, U = CAL.s_table(n / (s * s), t_nodes=(t,), s_nodes=(s,), epid=ep, seed=21)
    S, U = S / (s * s), U / (s * s)                 # back to per history
    prob = W.Problem(name="calib", phantom=CAL.slab_phantom(t), epid=ep, field=W.open_field(s, s),
                     lut=W.lut_table1(), physics=W.Physics(coupled=True), n_histories=n, seed=21)
    orc = oracle.run(prob)
    od, osd, _ = oracle.dose_stats(orc["tally"], n, ep)
    o_mean = od[mask].mean()
    # the oracle's region error from its own batches
    B = orc["tally"].shape[0]
    nb = oracle.batch_counts(n, B).astype(float)
    _, thick, rho = ep.layers[ep.sensitive]
    conv = 1.602176634e-13 / (rho * ep.pitch ** 2 * thick * 1e-3)
    per = orc["tally"][:, mask].mean(axis=1) * conv / nb
    o_sd = per.std(ddof=1) / np.sqrt(B)
    assert abs(S[0, 0] - o_mean) <= 3.0 * np.hypot(U[0, 0], o_sd)
    assert S[0, 0] == pytest.approx(o_mean, rel=0.01)         # same histories: replay
