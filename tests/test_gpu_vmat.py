"""GPU tests of VMAT arcs (control points as the fields of one batch), the
plan image (weighted sums of per-field dose and corrected signal) and the
resampling onto the 1190 x 1190 detector grid."""
import numpy as np
import pytest

import oracle
from tests import gpu_cases as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_24154_b300 import binding  # noqa: E402

STRIDE = 1 << 40


def _arc(n_cp, npx, pitch, seed=5):
    r = np.random.default_rng(seed)
    fields, mu = G.W.vmat_arc(r, n_cp)
    ph = G.W.thorax_ct(np.random.default_rng(1), 64, 64, 32, 0.8)
    ep = G.W.epid_default(npx, npx, pitch)
    p = G.W.Problem(name="vmat_small", phantom=ph, epid=ep, field=fields[0], lut=G.W.lut_bilinear(),
                    physics=G.W.Physics(coupled=True), n_histories=0, seed=seed)
    return p, fields, mu


def _sim(p, fields, **kw):
    sim = binding.Simulator(p.physics, **kw)
    sim.init_geometry(p.phantom, p.epid)
    sim.set_fields(fields, p.lut)
    return sim


def test_plan_image_equals_weighted_sum_of_fields():
    p, fields, mu = _arc(6, 96, 0.42)
    sim = _sim(p, fields)
    hist = [int(40_000 * 6 * m) + 1000 for m in mu]
    sim.run_batch(hist, p.seed)
    doses = [sim.dose(field=f)[0] for f in range(len(fields))]
    tmaps = [sim.tmap(field=f) for f in range(len(fields))]
    d, s = sim.plan_image(mu)
    wd, ws = oracle.plan_image(doses, tmaps, fields, p.lut, mu)
    assert np.allclose(d, wd, rtol=1e-12, atol=0)
    assert np.allclose(s, ws, rtol=1e-9, atol=1e-300)
    d_eq, _ = sim.plan_image(None)
    assert np.allclose(d_eq, sum(doses) / len(doses), rtol=1e-12, atol=0)


def test_vmat_arc_replays_oracle():
    p, fields, mu = _arc(8, 64, 0.6, seed=7)
    hist = [int(240_000 * m) for m in mu]
    sim = _sim(p, fields)
    st = sim.run_batch(hist, p.seed)
    assert G.energy_closure(st) < 2e-6
    d, _ = sim.plan_image(mu)
    orc_doses = []
    for f, fld in enumerate(fields):
        orc = oracle.run(p, n_histories=hist[f], hist_begin=f * STRIDE, field=fld)
        od, _, _ = oracle.dose_stats(orc["tally"], hist[f], p.epid)
        orc_doses.append(od)
        gt = sim.tally_all()[f].astype(np.float64) / G.QUANTA_PER_MEV
        assert gt.sum() == pytest.approx(orc["tally"].sum(), rel=1e-2), f
    od, _ = oracle.plan_image(orc_doses, [sim.tmap(field=f) for f in range(len(fields))], fields, p.lut, mu)
    assert d.sum() == pytest.approx(od.sum(), rel=5e-3)
    assert G.gamma_rate(od, d, p.epid.pitch, dd=0.02, dta_mm=2.0) >= 0.99


def test_resample_kernel_matches_oracle():
    r = np.random.default_rng(12)
    src = r.uniform(size=(160, 160))
    dst = torch.empty((1190, 1190), dtype=torch.float64, device="cuda:0")
    binding.resample_image(torch.tensor(src, device="cuda:0"), 0.25, dst, 0.0336)
    want = oracle.resample(src, 0.25, 1190, 1190, 0.0336)
    assert np.allclose(dst.cpu().numpy(), want, rtol=1e-12, atol=1e-15)


def test_vmat_on_the_1190_detector():
    """A 16-control-point arc on the thorax CT imaged by the 1190 x 1190,
    0.336 mm EPID: energy closure, every control point's image non-empty,
    the plan image finite."""
    ph, ep, fields, mu = G.W.config_vmat(n_cp=16, scale=2)
    p = G.W.Problem(name="vmat_1190", phantom=ph, epid=ep, field=fields[0], lut=G.W.lut_bilinear(),
                    physics=G.W.Physics(coupled=True), n_histories=0, seed=5)
    sim = _sim(p, fields, bank_capacity=1 << 22)
    hist = [int(4_000_000 * m) + 10_000 for m in mu]
    st = sim.run_batch(hist, p.seed)
    assert G.energy_closure(st) < 2e-6 and st["error_flags"] == 0
    tb = sim.tally_all()
    assert tb.shape == (16, 16, 1190, 1190)
    assert (tb.reshape(16, -1).sum(axis=1) > 0).all()
    d, s = sim.plan_image(mu)
    assert np.isfinite(d).all() and np.isfinite(s).all() and d.max() > 0
