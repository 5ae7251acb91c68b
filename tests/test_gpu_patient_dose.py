"""GPU tests of the patient dose tally (energy per CT voxel from the same
transport): closure with the CT energy counter, replay parity with the FP64
oracle's voxel tally, the analytic first-collision profile of a pencil beam,
and checkpoint/resume."""
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

J_PER_MEV = 1.602176634e-13


def _energy_mev(dose, phantom, n):
    rho, _ = oracle.hu_to_rho_mat(phantom.hu)
    return dose * rho.reshape(dose.shape) * np.prod(phantom.vox) * 1e-3 / J_PER_MEV * n


def test_voxel_tally_closes_with_ct_energy():
    p = G.thorax_case(n=50_000, scale=4, epid_scale=8)
    sim, st, _ = G.gpu_run(p, patient_dose=1)
    e = _energy_mev(sim.patient_dose(), p.phantom, st["histories"])
    # both are sums of the same 2^-8 eV quanta; the dose divides by the
    # float32 density the transport uses (relative rounding <= 6e-8)
    assert e.sum() == pytest.approx(st["e_ct"], rel=1e-7)
    assert (e >= 0).all()


def test_voxel_tally_replays_oracle():
    p = G.thorax_case(n=100_000, scale=4, epid_scale=8)
    sim, st, _ = G.gpu_run(p, patient_dose=1)
    orc = oracle.run(p, patient_dose=True)
    g = _energy_mev(sim.patient_dose(), p.phantom, st["histories"])
    o = orc["vox"]
    assert g.sum() == pytest.approx(o.sum(), rel=2e-3)
    # depth profile along the beam (+y at gantry 0) and the lateral profile
    for axes in ((0, 2), (0, 1)):
        gp, op = g.sum(axis=axes), o.sum(axis=axes)
        sel = op > 0.1 * op.max()
        assert np.allclose(gp[sel], op[sel], rtol=0.01), np.max(np.abs(gp[sel] / op[sel] - 1))


def test_pencil_beam_first_collision_profile():
    n = 2_000_000
    p = G.W.config_water_open(n_histories=n, field_cm=0.1)
    p.physics = G.W.Physics(coupled=False, mono_energy=1.0, photon_cutoff=0.999)
    sim, st, _ = G.gpu_run(p, patient_dose=1)
    depth = _energy_mev(sim.patient_dose(), p.phantom, n).sum(axis=(0, 2))
    out = (C.c_double * 3)()
    oracle.lib().orc_mu_photon(G.W.MAT_WATER, 1.0, out)
    mu = sum(out) * 1.0                      # water, density 1
    y = np.arange(depth.size + 1) * p.phantom.vox[1]
    want = n * (np.exp(-mu * y[:-1]) - np.exp(-mu * y[1:]))
    sd = np.sqrt(want * (1.0 - want / n))
    # single precision attenuation data: allow 0.3 % systematic on top of 4 sigma
    assert np.all(np.abs(depth - want) <= 4.0 * sd + 0.003 * want), np.max(np.abs(depth - want) / sd)


def test_patient_dose_checkpoint_resume():
    p = G.thorax_case(n=40_000, scale=4, epid_scale=8)
    a = G.make_sim(p, patient_dose=1)
    a.run(40_000, p.seed)
    whole = a.patient_dose()
    b = G.make_sim(p, patient_dose=1)
    b.run(15_000, p.seed)
    blob = b.get_state()
    c = G.make_sim(p, patient_dose=1)
    c.set_state(blob)
    c.run(25_000, p.seed)
    assert np.array_equal(c.patient_dose(), whole)
    off = G.make_sim(p)
    with pytest.raises(binding.MCError):
        off.patient_dose()
    with pytest.raises(binding.MCError):
        off.set_state(blob)             # a state with a voxel tally into a context without one
