"""GPU tests of batched multi-field runs (several static fields of one plan in
one wave sequence, Sec. 2.3's 25-field IMRT plan) and of the graph-driven
wave loop.

Field f of a batch draws from the random streams of a single-field run whose
history ids start at f * 2^40, and its tally lands in its own slice, so:
  * a batch's per-field tallies equal single-field runs bit for bit;
  * the graph-driven loop (one launch, device-side while-node) equals the
    host-driven loop bit for bit;
  * each field replays the oracle run with the same history ids.
"""
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


def _plan(n_fields=3, hist_lo=2e4, hist_hi=6e4, seed=2):
    ph, ep, fields, hist = G.W.config_batched_plan(seed=seed, n_fields=n_fields, scale=4, epid_scale=8,
                                                  hist_lo=hist_lo, hist_hi=hist_hi)
    p = G.W.Problem(name="batch_small", phantom=ph, epid=ep, field=fields[0], lut=G.W.lut_bilinear(),
                    physics=G.W.Physics(coupled=True), n_histories=hist[0], seed=seed)
    return p, fields, hist


def _batch_sim(p, fields, **overrides):
    sim = binding.Simulator(p.physics, **overrides)
    sim.init_geometry(p.phantom, p.epid)
    sim.set_fields(fields, p.lut)
    return sim


def test_batch_equals_single_field_runs_bitwise():
    p, fields, hist = _plan()
    sim = _batch_sim(p, fields)
    st = sim.run_batch(hist, p.seed)
    assert st["error_flags"] == 0 and st["histories"] == sum(hist)
    assert G.energy_closure(st) < 2e-6
    tb = sim.tally_all()
    counters = {k: 0 for k in oracle.COUNTER_NAMES}
    for f, fld in enumerate(fields):
        one = binding.Simulator(p.physics)
        one.init_geometry(p.phantom, p.epid)
        one.set_field(fld, p.lut)
        one.set_history_base(f * STRIDE)
        s1 = one.run(hist[f], p.seed)
        assert np.array_equal(tb[f], one.tally()), f
        for k in counters:
            counters[k] += s1["counters"][k]
        one.close()
    for k in oracle.COUNTER_NAMES:
        assert st["counters"][k] == counters[k], k


def test_graph_loop_equals_host_loop():
    p, fields, hist = _plan(seed=5)
    a = _batch_sim(p, fields, use_graph=0)
    sa = a.run_batch(hist, p.seed)
    b = _batch_sim(p, fields, use_graph=1)
    sb = b.run_batch(hist, p.seed)
    assert sb["error_flags"] == 0
    assert np.array_equal(a.tally_all(), b.tally_all())
    for k in oracle.COUNTER_NAMES:
        assert sa["counters"][k] == sb["counters"][k], k
    assert sa["waves"] == sb["waves"]
    assert sb["launches"] == sa["launches"] + sb["waves"]      # plus one wave-end kernel per wave
    # a second graph run continues the history ids like a second host run
    a.run_batch(hist, p.seed)
    b.run_batch(hist, p.seed)
    assert np.array_equal(a.tally_all(), b.tally_all())


def test_graph_loop_many_waves_single_field():
    """Small banks force many waves through the device-side loop."""
    p = G.thorax_case(n=60_000, scale=4, epid_scale=8)
    _, st_h, t_h = G.gpu_run(p, bank_capacity=1 << 14, primaries_per_wave=1 << 12)
    _, st_g, t_g = G.gpu_run(p, bank_capacity=1 << 14, primaries_per_wave=1 << 12, use_graph=1)
    assert st_h["waves"] > 10
    assert st_g["waves"] == st_h["waves"]
    assert np.array_equal(t_h, t_g)


def test_batch_fields_replay_oracle():
    p, fields, hist = _plan(n_fields=3, hist_lo=6e4, hist_hi=6.1e4, seed=7)
    sim = _batch_sim(p, fields)
    st = sim.run_batch(hist, p.seed)
    assert G.energy_closure(st) < 2e-6 and st["counters"]["lost"] == 0
    tb = sim.tally_all().astype(np.float64) / G.QUANTA_PER_MEV
    for f, fld in enumerate(fields):
        orc = oracle.run(p, n_histories=hist[f], hist_begin=f * STRIDE, field=fld)
        assert tb[f].sum() == pytest.approx(orc["tally"].sum(), rel=4e-3), f
        gd, gs, _ = sim.dose(field=f)
        od, os_, _ = oracle.dose_stats(orc["tally"], hist[f], p.epid)
        assert G.gamma_rate(od, gd, p.epid.pitch) >= 0.99, f
        frac, _ = G.three_sigma_fraction(gd, gs, od, os_)
        assert frac >= 0.99, f


def test_batch_per_field_readouts():
    """t-map, Eq. 1, dose statistics and the k(t, s) image of every field
    against the oracle's closed-form steps on the GPU's own tallies."""
    p, fields, hist = _plan(n_fields=4, hist_lo=5e3, hist_hi=2e4, seed=11)
    sim = _batch_sim(p, fields)
    sim.run_batch(hist, p.seed)
    tb = sim.tally_all().astype(np.float64) / G.QUANTA_PER_MEV
    for f, fld in enumerate(fields):
        s, a, b = sim.field_size(field=f)
        assert s == pytest.approx(oracle.effective_field_size(fld), rel=1e-12)
        t_orc = oracle.tmap(p, field=fld)
        assert np.allclose(sim.tmap(field=f), t_orc, rtol=1e-5, atol=1e-5)
        d, sg, u = sim.dose(field=f)
        od, os_, ou = oracle.dose_stats(tb[f], hist[f], p.epid)
        assert np.allclose(d, od, rtol=1e-12, atol=0)
        assert np.allclose(sg, os_, rtol=1e-9, atol=1e-30)
        want = oracle.lut_k(p.lut, t_orc, oracle.effective_field_size(fld)) * od
        assert np.allclose(sim.epid_image(field=f), want, rtol=2e-6, atol=1e-30)


def test_batch_checkpoint_and_errors():
    p, fields, hist = _plan(n_fields=2, hist_lo=5e3, hist_hi=1e4, seed=13)
    whole = _batch_sim(p, fields)
    whole.run_batch([2 * h for h in hist], p.seed)
    part = _batch_sim(p, fields)
    part.run_batch(hist, p.seed)
    blob = part.get_state()
    resumed = _batch_sim(p, fields)
    resumed.set_state(blob)
    resumed.run_batch(hist, p.seed)
    assert np.array_equal(resumed.tally_all(), whole.tally_all())
    with pytest.raises(binding.MCError):
        resumed.dose(field=2)
    with pytest.raises(binding.MCError):
        resumed.set_fields([], p.lut)
    one = binding.Simulator(p.physics)
    one.init_geometry(p.phantom, p.epid)
    one.set_field(fields[0], p.lut)
    with pytest.raises(binding.MCError):
        one.set_state(blob)             # two-field state into a one-field context


def test_autotuned_settings_change_time_not_results(tmp_path):
    from paper_2510_24154_b300 import autotune
    p = G.thorax_case(n=40_000, scale=4, epid_scale=8)
    search = {"regs_variant": [(4, 4, 4, 4), (3, 3, 4, 4)], "use_graph": [0, 1]}
    e = autotune.autotune(p, n_histories=40_000, search=search, path=tmp_path / "t.json")
    assert e["histories_per_s"] > 0 and e["trials"] >= 3
    _, _, t_def = G.gpu_run(p)
    _, _, t_tuned = G.gpu_run(p, **autotune.overrides(e))
    assert np.array_equal(t_def, t_tuned)
