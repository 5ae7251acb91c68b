"""GPU test of the arithmetic peak probes (mc_probe_alu_peaks): every rate
is positive and none exceeds what the SM's units can issue at the maximum
clock (148 SMs, 4 schedulers of one warp instruction per clock)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_24154_b300 import binding  # noqa: E402


def test_probe_rates_within_hardware_bounds():
    r = binding.probe_alu_peaks(0, repeats=2)
    sms = r["sm_count"]
    assert sms > 0 and r["ms_total"] > 0
    f_max = 2.032e9 * 1.02                     # maximum SM clock, small margin
    issue = sms * 4 * 32 * f_max / 1e12         # T thread-instructions/s
    for k in ("ffma_tflops", "ffma2_tflops", "mufu_tops", "int_tinst", "mix_tinst"):
        assert r[k] > 0, k
    # one FMA is one thread-instruction; an f32x2 FMA does two per instruction
    assert r["ffma_tflops"] / 2 <= 2 * issue
    assert r["ffma2_tflops"] / 4 <= issue
    assert r["int_tinst"] <= issue and r["mix_tinst"] <= issue
    assert r["mufu_tops"] <= issue
    # the FMA pipe runs at a good part of its rate under this load
    assert r["ffma_tflops"] / 2 > 0.25 * issue


def test_probe_arguments_checked():
    with pytest.raises(binding.MCError):
        binding.probe_alu_peaks(0, repeats=0)
    with pytest.raises(binding.MCError):
        binding.probe_alu_peaks(10_000, repeats=1)
