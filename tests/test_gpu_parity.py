"""GPU parity tests: the CUDA path through the C-ABI against the FP64 oracle on
the same seeded inputs.

Transport is a stochastic estimator, so parity is checked in two tiers:
  replay       both sides use the same Philox keys and draw order, so each
               history is the same up to single- vs double-precision rounding;
               the images must pass a 1 %/1 mm global gamma (10 % threshold)
               with the oracle as reference at >= 99.5 % of pixels;
  independent  different seeds; per-pixel |D_gpu - D_orc| <= 3 sqrt(s_g^2 + s_o^2)
               for >= 99 % of pixels above 10 % of the maximum.
Integer and closed-form steps (Philox, the uniform stream, Eq. 1, dose
statistics from the integer tallies) are compared exactly or to FP64 rounding.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from tests import gpu_cases as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_24154_b300 import binding  # noqa: E402


# ------------------------------------------------------------ RNG -------

def test_philox_bit_exact():
    rng = np.random.default_rng(0)
    rows = rng.integers(0, 2 ** 32, size=(20000, 6), dtype=np.uint64).astype(np.uint32)
    rows[0] = 0
    rows[1] = 0xFFFFFFFF
    got = binding.test_philox(rows)
    lib = oracle.lib()
    for i in range(rows.shape[0]):
        out = (C.c_uint32 * 4)()
        lib.orc_philox((C.c_uint32 * 4)(*rows[i, :4]), (C.c_uint32 * 2)(*rows[i, 4:]), out)
        assert list(got[i]) == list(out)


@pytest.mark.parametrize("seed,hist,ord_", [(0, 0, 0), (1, 12345, 7), (2 ** 40 + 3, 2 ** 33 + 5, 0xDEADBEEF)])
def test_uniform_stream_bit_exact(seed, hist, ord_):
    n = 67
    g = binding.test_uniforms(seed, hist, ord_, n).astype(np.float64)
    o = np.empty(n)
    oracle.lib().orc_uniforms(seed, hist, ord_, n, o.ctypes.data_as(C.POINTER(C.c_double)))
    assert np.array_equal(g, o)


# ------------------------------------------------- closed-form steps ----

def test_eq1_field_size_and_tmap_small():
    p = G.thorax_case(scale=4, epid_scale=8)
    sim = G.make_sim(p)
    s, a, b = sim.field_size()
    oa, ob = oracle.aperture_bbox(p.field)
    assert (a, b) == pytest.approx((oa, ob), rel=1e-12)
    assert s == pytest.approx(oracle.effective_field_size(p.field), rel=1e-12)
    t_gpu = sim.tmap()
    t_orc = oracle.tmap(p)
    assert np.allclose(t_gpu, t_orc, rtol=1e-5, atol=1e-5)
    assert t_orc.max() > 10.0


@pytest.mark.parametrize("gantry", [0.0, 37.0, 90.0, 211.5])
def test_tmap_gantry_angles(gantry):
    p = G.thorax_case(scale=4, epid_scale=8, gantry=gantry)
    sim = G.make_sim(p)
    assert np.allclose(sim.tmap(), oracle.tmap(p), rtol=1e-5, atol=1e-5)


def test_tmap_full_size_sampled_pixels():
    p = G.thorax_case(scale=1, epid_scale=1)
    sim = G.make_sim(p)
    t_gpu = sim.tmap()
    rng = np.random.default_rng(3)
    iy = rng.integers(0, p.epid.npy, 600)
    ix = rng.integers(0, p.epid.npx, 600)
    t_orc = oracle.tmap(p, ix, iy)
    assert np.allclose(t_gpu[iy, ix], t_orc, rtol=1e-5, atol=1e-5)


def test_dose_stats_and_lut_from_gpu_tally():
    """Dose statistics and the k(t, s) correction on the GPU's own integer tally: dose and sigma to FP64
    rounding, signal to float32 rounding of k(t, s) * dose."""
    for lut in (G.W.lut_bilinear(), G.W.lut_wavy(), G.W.lut_table1()):
        p = G.thorax_case(n=20_000, scale=4, epid_scale=8)
        p.lut = lut
        sim, st, tally = G.gpu_run(p)
        d, s, u = sim.dose()
        od, os_, ou = oracle.dose_stats(tally, st["histories"], p.epid)
        assert np.allclose(d, od, rtol=1e-12, atol=0)
        assert np.allclose(s, os_, rtol=1e-9, atol=1e-30)
        assert u == pytest.approx(ou, rel=1e-9)
        sig = sim.epid_image()
        want = oracle.lut_k(lut, oracle.tmap(p), oracle.effective_field_size(p.field)) * od
        assert np.allclose(sig, want, rtol=2e-6, atol=1e-30)


# ------------------------------------------------------- transport ------

def _compare_replay(p, n, gpu_seed=None):
    sim, st, gt = G.gpu_run(p, n=n, seed=gpu_seed)
    orc = oracle.run(p, n_histories=n)
    ot = orc["tally"]
    assert G.energy_closure(st) < 2e-6, st
    assert st["counters"]["lost"] == 0 and st["error_flags"] == 0
    e_g, e_o = gt.sum(), ot.sum()
    gd, gs, _ = sim.dose()
    od, os_, _ = oracle.dose_stats(ot, n, p.epid)
    return sim, st, orc, gt, ot, (e_g, e_o), (gd, gs, od, os_)


def test_replay_photon_only_water():
    """The small single-field workload on its exact grid: photon-only, 1e6
    histories, water box of 64 x 40 x 64 at 5 mm, open 10 x 10 field, EPID
    128 x 128 at 3 mm."""
    p = G.water_case(n=1_000_000, coupled=False, npx=128, pitch=0.3)
    sim, st, orc, gt, ot, (e_g, e_o), (gd, gs, od, os_) = _compare_replay(p, p.n_histories)
    assert abs(e_g / e_o - 1) < 1e-4
    for k in ("flights_ct", "real_ct", "compton", "photo", "pair", "primaries_at_epid", "uncollided_at_epid"):
        assert st["counters"][k] == pytest.approx(orc["counters"][k], rel=1e-4), k
    assert G.gamma_rate(od, gd, p.epid.pitch) >= 0.995
    frac, npx_sel = G.three_sigma_fraction(gd, gs, od, os_)
    assert frac >= 0.99 and npx_sel > 100


def test_replay_coupled_thorax():
    p = G.thorax_case(n=200_000, scale=4, epid_scale=8)
    sim, st, orc, gt, ot, (e_g, e_o), (gd, gs, od, os_) = _compare_replay(p, p.n_histories)
    assert abs(e_g / e_o - 1) < 2e-3
    for k in ("flights_ct", "real_ct", "compton", "esteps_ct", "esteps_epid", "electrons", "moller", "brem"):
        assert st["counters"][k] == pytest.approx(orc["counters"][k], rel=2e-3), k
    assert G.gamma_rate(od, gd, p.epid.pitch) >= 0.995
    frac, _ = G.three_sigma_fraction(gd, gs, od, os_)
    assert frac >= 0.99


@pytest.mark.parametrize("case", ["water_photon", "water_coupled", "thorax"])
def test_independent_streams_three_sigma(case):
    if case == "water_photon":
        p = G.water_case(n=2_000_000, coupled=False, batches=64)
    elif case == "water_coupled":
        p = G.water_case(n=400_000, coupled=True, batches=64)
    else:
        p = G.thorax_case(n=400_000, scale=4, epid_scale=8, batches=64)
    sim, st, gt = G.gpu_run(p, seed=p.seed + 1000)
    orc = oracle.run(p)
    gd, gs, _ = sim.dose()
    od, os_, _ = oracle.dose_stats(orc["tally"], p.n_histories, p.epid)
    frac, nsel = G.three_sigma_fraction(gd, gs, od, os_)
    assert nsel > 200
    assert frac >= 0.99, (frac, nsel)


def test_full_size_thorax_replay_pixel_by_pixel():
    """The full thorax workload (CT 256 x 256 x 128 at 2 mm, EPID 1024 x 768 at
    0.39 mm, 9-segment field, coupled) in bench.py's launch configuration,
    replayed against the oracle pixel by pixel on the full detector grid: a
    1 %/1 mm global gamma (10 % threshold) with the oracle's image as
    reference passes at >= 98.5 % of pixels (measured 99.1 %).

    Why not 99.5 % here: at 1e6 histories on 0.39 mm pixels the image is
    sparse (a pixel above the threshold holds one or two tracks), so each
    history that FP32 rounding takes off its FP64 path fails its own one to
    three pixels outright.  Bisecting 65,536 histories one by one found 8
    whose image differs by more than 1e-3 anywhere: 6 split a layer crossing's
    energy differently by ~1e-3 (same pixels), 2 put a deposit 1-3 pixels
    away (a bremsstrahlung photon and a long electron track, whose direction
    differences grow over the ~60 cm to the detector), i.e. ~3e-5 of
    histories; each side is bitwise the same when the run is split."""
    n = 1_000_000
    p = G.thorax_case(n=n, scale=1, epid_scale=1)
    sim, st, gt = G.gpu_run(p, bank_capacity=1 << 26)
    orc = oracle.run(p)
    assert G.energy_closure(st) < 2e-6 and st["error_flags"] == 0 and st["counters"]["lost"] == 0
    gd, _, _ = sim.dose()
    od, _, _ = oracle.dose_stats(orc["tally"], n, p.epid)
    assert gd.shape == (768, 1024)
    assert (od > 0.1 * od.max()).sum() > 2000
    assert gt.sum() == pytest.approx(orc["tally"].sum(), rel=1e-3)
    rate = G.gamma_rate(od, gd, p.epid.pitch)
    assert rate >= 0.985, rate


def test_full_size_geometry_replay():
    """The full thorax CT (256x256x128 at 2 mm) and EPID (1024x768 at 0.39 mm)
    in the default launch configuration: energy balance, replay of the
    sensitive-layer energy and of the event counts."""
    p = G.thorax_case(n=200_000, scale=1, epid_scale=1)
    sim, st, gt = G.gpu_run(p, bank_capacity=1 << 26)       # bench.py's launch configuration
    orc = oracle.run(p)
    assert G.energy_closure(st) < 2e-6
    assert gt.sum() == pytest.approx(orc["tally"].sum(), rel=5e-3)
    for k in ("real_ct", "compton", "electrons", "primaries_at_epid"):
        assert st["counters"][k] == pytest.approx(orc["counters"][k], rel=2e-3), k


def test_bench_step_statistics_against_oracle_sample():
    """The benchmark step itself (full thorax CT and EPID, 1e8 histories,
    2^26-particle banks): energy balance, no lost particles, and the mean
    sensitive-layer energy and event counts per history within 4 standard
    errors of an independent oracle sample of 4e5 histories, run as 16 chunks
    of 25,000 whose spread gives each quantity's standard error (the GPU's
    own error is 16x smaller)."""
    n_gpu, n_chunk, n_ch = 100_000_000, 25_000, 16
    p = G.thorax_case(n=n_gpu, scale=1, epid_scale=1, batches=16)
    sim, st, gt = G.gpu_run(p, bank_capacity=1 << 26)
    assert st["histories"] == n_gpu and st["error_flags"] == 0 and st["counters"]["lost"] == 0
    assert G.energy_closure(st) < 2e-6
    keys = ("flights_ct", "real_ct", "compton", "esteps_ct", "electrons", "primaries_at_epid")
    per = {k: [] for k in keys + ("sensitive",)}
    for c in range(n_ch):                     # streams disjoint from the GPU's
        orc = oracle.run(p, n_histories=n_chunk, hist_begin=(1 << 40) + c * n_chunk)
        per["sensitive"].append(orc["tally"].sum() / n_chunk)
        for k in keys:
            per[k].append(orc["counters"][k] / n_chunk)
    got = {"sensitive": gt.sum() / n_gpu}
    got.update({k: st["counters"][k] / n_gpu for k in keys})
    for k, v in per.items():
        v = np.asarray(v)
        se = v.std(ddof=1) / np.sqrt(n_ch)
        assert abs(got[k] - v.mean()) <= 4.0 * se, (k, got[k], v.mean(), se)


# --------------------------------------------------- determinism --------

def test_bitwise_reproducible_across_runs_and_launch_shapes():
    p = G.thorax_case(n=100_000, scale=4, epid_scale=8)
    _, st1, t1 = G.gpu_run(p)
    _, st2, t2 = G.gpu_run(p)
    _, st3, t3 = G.gpu_run(p, block_size=128, bank_capacity=1 << 18, primaries_per_wave=1 << 14)
    # a wave size far above the bank: each wave admits at most half a bank
    _, st4, t4 = G.gpu_run(p, bank_capacity=1 << 14, primaries_per_wave=1 << 22)
    assert np.array_equal(t1, t2) and np.array_equal(t1, t3) and np.array_equal(t1, t4)
    assert st4["error_flags"] == 0 and st4["waves"] > st1["waves"]
    physics = oracle.COUNTER_NAMES          # the execution counters depend on the launch shape
    assert all(st1["counters"][k] == st3["counters"][k] == st4["counters"][k] for k in physics)
    assert st1["e_src"] == st3["e_src"] == st4["e_src"] and st1["e_ct"] == st3["e_ct"] == st4["e_ct"]
    # per-layer EPID energy (lanes hold pending deposits; the many-wave run
    # defers its EPID electrons to the last source wave)
    assert np.array_equal(st1["e_epid"], st3["e_epid"]) and np.array_equal(st1["e_epid"], st4["e_epid"])


def test_checkpoint_resume_is_bitwise_identical():
    p = G.thorax_case(n=60_000, scale=4, epid_scale=8)
    sim_a = G.make_sim(p)
    sim_a.run(60_000, p.seed)
    whole = sim_a.tally()
    sim_b = G.make_sim(p)
    sim_b.run(25_000, p.seed)
    blob = sim_b.get_state()
    sim_c = G.make_sim(p)
    sim_c.set_state(blob)
    sim_c.run(35_000, p.seed)
    assert np.array_equal(sim_c.tally(), whole)
    assert sim_c.stats()["histories"] == 60_000


def test_split_runs_equal_one_run():
    p = G.water_case(n=300_000, coupled=True)
    sim = G.make_sim(p)
    sim.run(100_000, p.seed)
    sim.run(200_000, p.seed)
    _, _, t_one = G.gpu_run(p)
    assert np.array_equal(sim.tally().astype(np.float64) / G.QUANTA_PER_MEV, t_one)


def test_input_errors_are_reported():
    p = G.water_case(n=10)
    from paper_2510_24154_b300.binding import MCError, Simulator
    sim = Simulator(p.physics)
    with pytest.raises(MCError):
        sim.run(10, 0)                       # no geometry / field yet
    sim.init_geometry(p.phantom, p.epid)
    bad = G.W.open_field(10, 10)
    bad.mu = np.array([0.0])
    with pytest.raises(MCError):
        sim.set_field(bad)
    closed = G.W.open_field(10, 10)
    closed.sid = 60.0                         # detector inside the CT
    with pytest.raises(MCError):
        sim.set_field(closed)


def test_replay_with_leaf_transmission():
    """Leaf transmission (1.5 %) in both source models: the primaries behind
    closed leaves replay like the others."""
    p = G.thorax_case(n=200_000, scale=4, epid_scale=8)
    p.field.leaf_transmission = 0.015
    sim, st, orc, gt, ot, (e_g, e_o), (gd, gs, od, os_) = _compare_replay(p, p.n_histories)
    assert abs(e_g / e_o - 1) < 2e-3
    assert G.gamma_rate(od, gd, p.epid.pitch) >= 0.995
    frac, _ = G.three_sigma_fraction(gd, gs, od, os_)
    assert frac >= 0.99
    q = G.thorax_case(n=200_000, scale=4, epid_scale=8)
    _, _, g0 = G.gpu_run(q)
    # behind the leaves (pixels below 2 % of the open-field maximum without
    # transmission) the signal grows; histories are redistributed, so the
    # total need not
    img0, img1 = g0.sum(axis=0), gt.sum(axis=0)
    low = img0 < 0.02 * img0.max()
    assert low.sum() > 100 and img1[low].sum() > 1.5 * img0[low].sum()


def test_replay_with_collimation():
    """Leaf and jaw transmission, tongue and groove, leaf gap: both source
    builders must produce the same rectangles in the same order, so a
    photon-only run replays the oracle pixel by pixel (an independent stream
    would differ by its full noise, tens of per cent per pixel)."""
    p = G.thorax_case(n=400_000, scale=4, epid_scale=8)
    p.physics.coupled = False
    f = p.field
    f.leaf_transmission, f.jaw_transmission, f.tg_width, f.leaf_gap = 0.015, 0.005, 0.1, 0.15
    sim, st, orc, gt, ot, (e_g, e_o), (gd, gs, od, os_) = _compare_replay(p, p.n_histories)
    assert abs(e_g / e_o - 1) < 1e-3
    for k in ("flights_ct", "real_ct", "compton", "primaries_at_epid", "uncollided_at_epid"):
        assert st["counters"][k] == pytest.approx(orc["counters"][k], rel=5e-4), k
    assert G.gamma_rate(od, gd, p.epid.pitch) >= 0.995
    frac, nsel = G.three_sigma_fraction(gd, gs, od, os_)
    assert frac >= 0.99 and nsel > 200


def test_collimation_arguments_rejected():
    p = G.thorax_case(n=1000, scale=4, epid_scale=8)
    for name, v in (("jaw_transmission", 1.0), ("tg_width", 0.6), ("leaf_gap", 2.0), ("leaf_transmission", -0.1)):
        q = G.thorax_case(n=1000, scale=4, epid_scale=8)
        setattr(q.field, name, v)
        with pytest.raises(binding.MCError):
            G.make_sim(q)
    G.make_sim(p).close()


def test_replay_with_collimator_slabs():
    """Leaves (6 cm) and jaws (7.8 cm) as tungsten slabs: both sides draw the
    same source photons until one leaves the collimators (phase space 2),
    transport it through the slabs the same way and then through the
    patient; coupled replay against the oracle (energy, counters, 1 %/1 mm
    gamma >= 99.5 %, 3 sigma >= 99 %), and behind closed leaves the signal is
    the tungsten's transmission, not zero."""
    p = G.thorax_case(n=200_000, scale=4, epid_scale=8)
    p.field.leaf_thickness, p.field.jaw_thickness = 6.0, 7.8
    sim, st, orc, gt, ot, (e_g, e_o), (gd, gs, od, os_) = _compare_replay(p, p.n_histories)
    assert abs(e_g / e_o - 1) < 2e-3
    for k in ("flights_ct", "real_ct", "compton", "esteps_ct", "electrons", "primaries_at_epid", "uncollided_at_epid"):
        assert st["counters"][k] == pytest.approx(orc["counters"][k], rel=2e-3), k
    assert G.gamma_rate(od, gd, p.epid.pitch) >= 0.995
    frac, _ = G.three_sigma_fraction(gd, gs, od, os_)
    assert frac >= 0.99
    q = G.thorax_case(n=200_000, scale=4, epid_scale=8)
    _, _, g0 = G.gpu_run(q)
    img0, img1 = g0.sum(axis=0), gt.sum(axis=0)
    low = img0 < 0.02 * img0.max()
    assert low.sum() > 100 and img1[low].sum() > 1.5 * img0[low].sum()


def test_slab_source_photon_only_replay_and_transmission():
    """Photon-only, the slab source on the water workload with every leaf
    closed but a 4 x 4 cm opening (1 cm tungsten leaves, 2 MeV photons, the
    water box moved off the beam): the counts of primaries reaching the EPID
    and of those unscattered replay the oracle exactly up to FP32 rounding,
    and the unscattered share behind the leaves is the slab's transmission."""
    from tests.test_oracle_pins import _slab_field
    p = G.water_case(n=400_000, coupled=False)
    p.field = _slab_field((-2.0, 2.0, -2.0, 2.0), leaf_t=1.0)
    p.physics.mono_energy = 2.0
    ph = p.phantom
    p.phantom = G.W.Phantom(ph.hu, ph.vox, (ph.origin[0] + 40.0, ph.origin[1], ph.origin[2]))
    sim, st, gt = G.gpu_run(p)
    orc = oracle.run(p)
    assert G.energy_closure(st) < 2e-6 and st["error_flags"] == 0
    for k in ("primaries_at_epid", "uncollided_at_epid", "flights_epid", "compton", "photo"):
        assert st["counters"][k] == pytest.approx(orc["counters"][k], rel=1e-3), k
    assert gt.sum() == pytest.approx(orc["tally"].sum(), rel=1e-3)
