"""GPU tests at the full size of the anthropomorphic workload: a 512 x 512 x 200
HU phantom at 1 mm, one 40-segment IMRT field, the 1190 x 1190 EPID at
0.336 mm.  Replay against the FP64 oracle on a sample of histories (pixel by
pixel on the full detector grid), the
radiological thickness of sampled pixels against the oracle's ray sums, and
the properties of a 2e8-history run (energy closure, no lost particles, the
statistics falling as 1/sqrt(N))."""
import numpy as np
import pytest

import oracle
from tests import gpu_cases as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def problem():
    return G.W.config_anthropomorphic(n_histories=200_000)


def test_replay_sample_of_histories(problem):
    p = problem
    n = 200_000
    sim, st, gt = G.gpu_run(p, n=n)
    orc = oracle.run(p, n_histories=n)
    ot = orc["tally"]
    assert G.energy_closure(st) < 2e-6 and st["error_flags"] == 0 and st["counters"]["lost"] == 0
    assert gt.sum() == pytest.approx(ot.sum(), rel=3e-3)
    # counters: FP32 rounding lets a few per cent of histories leave the
    # replay at 1 mm voxels; those differ by their own noise
    for k in ("flights_ct", "real_ct", "compton", "esteps_ct", "esteps_epid", "electrons", "primaries_at_epid"):
        g, o = st["counters"][k], orc["counters"][k]
        assert abs(g - o) <= 3e-3 * o + 5.0 * np.sqrt(o), (k, g, o)
    # pixel by pixel on the full 1190 x 1190 grid: 1 %/1 mm global gamma with
    # the oracle's image as reference, >= 98 % (measured 98.9 %; on this
    # sparse image every history that rounding takes off its FP64 path fails
    # its own few pixels, as in the thorax full-grid replay)
    gd, _, _ = sim.dose()
    od, _, _ = oracle.dose_stats(ot, n, p.epid)
    assert gd.shape == (1190, 1190)
    assert (od > 0.1 * od.max()).sum() > 1000
    rate = G.gamma_rate(od, gd, p.epid.pitch)
    assert rate >= 0.98, rate
    sim.close()


def test_tmap_sampled_pixels(problem):
    p = problem
    sim = G.make_sim(p)
    t = sim.tmap()
    r = np.random.default_rng(3)
    ix = r.integers(0, p.epid.npx, 300)
    iy = r.integers(0, p.epid.npy, 300)
    want = oracle.tmap(p, ix, iy)
    assert np.allclose(t[iy, ix], want, rtol=1e-5, atol=2e-5)
    assert want.max() > 20.0                      # rays cross the body
    sim.close()


def _binned_u(tally):
    """Mean relative batch error over 16 x 16-pixel bins above half the
    maximum (5.4 mm bins hold enough deposits for the 1/sqrt(N) law)."""
    t = tally.astype(np.float64)[:, :1184, :1184]
    B = t.shape[0]
    t = t.reshape(B, 74, 16, 74, 16).sum(axis=(2, 4))
    m = t.mean(axis=0)
    s = t.std(axis=0, ddof=1) / np.sqrt(B)
    sel = m > 0.5 * m.max()
    return float(np.mean(s[sel] / m[sel]))


def test_full_size_run_properties(problem):
    p = problem
    sim = G.make_sim(p)
    sim.run(50_000_000, p.seed)
    _, _, u1 = sim.dose()
    ub1 = _binned_u(sim.tally())
    st = sim.run(150_000_000, p.seed)
    assert st["histories"] == 200_000_000
    assert G.energy_closure(st) < 2e-6 and st["error_flags"] == 0 and st["counters"]["lost"] == 0
    d, s, u = sim.dose()
    assert np.isfinite(d).all() and d.max() > 0 and (s >= 0).all()
    # per 0.336 mm pixel the counts are still small (u ~ 0.4-0.6), where the
    # batch estimate falls more slowly than 1/sqrt(N); binned, four times the
    # histories halve the relative uncertainty
    assert u < u1
    assert _binned_u(sim.tally()) == pytest.approx(ub1 / 2.0, rel=0.1)
    img = sim.epid_image()
    assert np.isfinite(img).all() and img.max() > 0
    sim.close()
