"""The allocation-free dose-statistics entry point against mc_get_dose.

mc_dose_stats_noalloc is for callers that may not allocate device memory
while running (a service whose framework allocator already owns the GPU's
memory, or software whose rules forbid run-time allocation).  It keeps its
scratch in a fixed array inside the library, shared by every call, so this
test makes two calls in a row on different images, the second with a smaller
maximum and a different size, and checks each against the context-based
mc_get_dose of the same tally.  It lives in its own file, collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_24154_b300 import binding, workloads as W  # noqa: E402


def _case(problem, n):
    """Run `problem` through the context path; return its tally on the device,
    the pixel mass and mc_get_dose's (dose, sigma, u)."""
    sim = binding.Simulator(problem.physics)
    sim.init_geometry(problem.phantom, problem.epid)
    sim.set_field(problem.field, problem.lut)
    sim.run(n, problem.seed)
    dose, sigma, u = sim.dose()
    tally = torch.from_numpy(sim.tally().view(np.int64)).cuda()
    _, thick, rho = problem.epid.layers[problem.epid.sensitive]
    pitch = problem.epid.pitch
    mass_kg = rho * pitch * pitch * thick * 1e-3
    sim.close()
    return tally, mass_kg, (dose, sigma, u)


def test_noalloc_matches_mc_get_dose_on_two_calls_in_a_row():
    a = W.config_thorax_imrt(n_histories=40_000, scale=4, epid_scale=8)
    b = W.config_water_open(n_histories=200_000, npx=64, npy=48, pitch=0.6)
    cases = [(a, 40_000), (b, 200_000)]
    prepared = [_case(p, n) for p, n in cases]
    # larger image maximum first: a maximum left over in the shared scratch
    # would then spoil the second call's threshold for u
    order = sorted(range(2), key=lambda i: -prepared[i][2][0].max())
    assert prepared[order[0]][2][0].max() > prepared[order[1]][2][0].max()
    for i in order:
        (p, n), (tally, mass, (d_ref, s_ref, u_ref)) = cases[i], prepared[i]
        ny, nx = p.epid.npy, p.epid.npx
        dose = torch.full((ny, nx), -1.0, dtype=torch.float64, device="cuda")
        sigma = torch.full((ny, nx), -1.0, dtype=torch.float64, device="cuda")
        u = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        binding.dose_stats_noalloc(tally, nx, ny, p.physics.n_batches, n, mass, dose, sigma, u)
        torch.cuda.synchronize()
        assert np.allclose(dose.cpu().numpy(), d_ref, rtol=1e-12, atol=0)
        assert np.allclose(sigma.cpu().numpy(), s_ref, rtol=1e-12, atol=1e-300)
        assert float(u.item()) == pytest.approx(u_ref, rel=1e-12)


def test_noalloc_dose_only_and_the_batch_limit():
    """A dose-only call (no sigma, no u) and a call at the largest batch count
    (1024), each against mc_get_dose of the same tally."""
    p = W.config_water_open(n_histories=100_000, npx=24, npy=16, pitch=1.0)
    p.physics.n_batches = 1024
    tally, mass, (d_ref, s_ref, u_ref) = _case(p, 100_000)
    ny, nx = p.epid.npy, p.epid.npx
    dose = torch.full((ny, nx), -1.0, dtype=torch.float64, device="cuda")
    binding.dose_stats_noalloc(tally, nx, ny, 1024, 100_000, mass, dose)
    torch.cuda.synchronize()
    assert np.allclose(dose.cpu().numpy(), d_ref, rtol=1e-12, atol=0)
    sigma = torch.full((ny, nx), -1.0, dtype=torch.float64, device="cuda")
    u = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    binding.dose_stats_noalloc(tally, nx, ny, 1024, 100_000, mass, dose, sigma, u)
    torch.cuda.synchronize()
    assert np.allclose(dose.cpu().numpy(), d_ref, rtol=1e-12, atol=0)
    assert np.allclose(sigma.cpu().numpy(), s_ref, rtol=1e-12, atol=1e-300)
    assert float(u.item()) == pytest.approx(u_ref, rel=1e-12)


def test_noalloc_rejects_bad_inputs():
    t = torch.zeros(64, dtype=torch.int64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.MCError):       # more pixels than the scratch holds
        binding.dose_stats_noalloc(t, 4096, 2048, 16, 100, 1e-6, out)
    with pytest.raises(binding.MCError):       # more batches than the scratch holds
        binding.dose_stats_noalloc(t, 2, 2, 2048, 100_000, 1e-6, out)
    with pytest.raises(binding.MCError):       # fewer histories than batches: empty batches
        binding.dose_stats_noalloc(t, 2, 2, 16, 15, 1e-6, out)
