"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads, and
exports every entry point include/archer_epid.h and include/archer_denoise.h
declare; the ctypes struct mirrors match the C layout.  No compute call is
made (no GPU here)."""
import ctypes as C
import re
import subprocess
import textwrap
from pathlib import Path

import pytest

from paper_2510_24154_b300 import binding, build, denoise

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "archer_epid.h"
DN_HEADER = ROOT / "include" / "archer_denoise.h"


def declared_entry_points(header=HEADER, prefix="mc_"):
    text = header.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(" + prefix + r"[a-z_0-9]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert declared_entry_points() == sorted(binding.EXPORTED)
    assert declared_entry_points(DN_HEADER, "dn_") == sorted(denoise.EXPORTED)


def test_library_builds_and_exports_every_symbol():
    lib_path = build.build()
    assert lib_path.exists()
    out = subprocess.run(["nm", "-D", "--defined-only", str(lib_path)], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+((?:mc|dn)_\w+)", out))
    declared = set(declared_entry_points()) | set(declared_entry_points(DN_HEADER, "dn_"))
    missing = declared - exported
    assert not missing, f"missing exports: {missing}"
    lib = C.CDLL(str(lib_path))
    for name in declared:
        assert hasattr(lib, name)


def test_build_targets_sm103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_config_default_without_gpu():
    lib = binding.load()
    cfg = binding.Config()
    lib.mc_config_default(C.byref(cfg))
    assert cfg.coupled == 1 and cfg.n_batches == 16
    assert cfg.photon_cutoff_mev == pytest.approx(0.01) and cfg.electron_cutoff_mev == pytest.approx(0.2)
    assert lib.mc_status_string(8) == b"particle bank overflow"


def test_argument_errors_need_no_gpu():
    lib = binding.load()
    assert lib.mc_create(None, 0, None) == 1            # MC_ERR_ARG on a null out-pointer
    assert lib.mc_destroy(None) == 0
    assert lib.mc_cancel(None) == 1
    # the arithmetic peak probe checks its arguments before touching a device
    import ctypes as C
    r = binding.AluPeaks()
    assert lib.mc_probe_alu_peaks(0, 1, None) == 1
    assert lib.mc_probe_alu_peaks(0, 0, C.byref(r)) == 1
    assert lib.mc_probe_alu_peaks(0, 101, C.byref(r)) == 1
    assert lib.mc_probe_alu_peaks(-1, 1, C.byref(r)) == 1


def test_struct_layouts_match_c(tmp_path):
    probe = textwrap.dedent("""
        #include <stdio.h>
        #include <stddef.h>
        #include "archer_epid.h"
        #include "archer_denoise.h"
        int main(void) {
          printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(mc_config), sizeof(mc_epid_desc), sizeof(mc_field_desc),
                 sizeof(mc_lut_desc), sizeof(mc_run_stats), sizeof(mc_alu_peaks), offsetof(mc_alu_peaks, sm_count));
          printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", offsetof(mc_config, use_graph), offsetof(mc_config, regs_variant), offsetof(mc_config, patient_dose),
                 offsetof(mc_epid_desc, pitch_cm),
                 offsetof(mc_field_desc, eq1_literal), offsetof(mc_field_desc, leaf_transmission),
                 offsetof(mc_field_desc, leaf_gap_cm), offsetof(mc_run_stats, gpu_ms),
                 offsetof(mc_run_stats, launches));
          printf("%zu %zu\\n", offsetof(mc_field_desc, leaf_thickness_cm), offsetof(mc_field_desc, jaw_thickness_cm));
          printf("%zu %zu %zu\\n", sizeof(dn_config), offsetof(dn_config, in_channels), offsetof(dn_config, seed));
          return 0;
        }""")
    src = tmp_path / "probe.c"
    src.write_text(probe)
    exe = tmp_path / "probe"
    subprocess.run(["gcc", f"-I{ROOT / 'include'}", str(src), "-o", str(exe)], check=True)
    sizes, offs, slabs, dn = [list(map(int, l.split())) for l in
                              subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()]
    assert slabs == [binding.FieldDesc.leaf_thickness_cm.offset, binding.FieldDesc.jaw_thickness_cm.offset]
    assert dn == [C.sizeof(denoise.DnConfig), denoise.DnConfig.in_channels.offset, denoise.DnConfig.seed.offset]
    assert sizes == [C.sizeof(binding.Config), C.sizeof(binding.EpidDesc), C.sizeof(binding.FieldDesc),
                     C.sizeof(binding.LutDesc), C.sizeof(binding.RunStats), C.sizeof(binding.AluPeaks),
                     binding.AluPeaks.sm_count.offset]
    assert offs == [binding.Config.use_graph.offset, binding.Config.regs_variant.offset, binding.Config.patient_dose.offset, binding.EpidDesc.pitch_cm.offset,
                    binding.FieldDesc.eq1_literal.offset, binding.FieldDesc.leaf_transmission.offset,
                    binding.FieldDesc.leaf_gap_cm.offset, binding.RunStats.gpu_ms.offset,
                    binding.RunStats.launches.offset]


def test_denoise_config_layout_and_errors_without_gpu():
    probe_ok = denoise.DnConfig()
    lib = denoise.lib()
    lib.dn_config_default(C.byref(probe_ok))
    assert (probe_ok.height, probe_ok.width, probe_ok.levels, probe_ok.base_channels, probe_ok.in_channels) == \
        (768, 1024, 4, 32, 1)
    assert lib.dn_create(None, 0, None) == 1
    bad = denoise.DnConfig(height=100, width=1024, batch=1, levels=4, base_channels=32, seed=0)   # not a multiple of 8
    h = C.c_void_p()
    assert lib.dn_create(C.byref(bad), 0, C.byref(h)) == 1 and not h.value
    for planes in (0, 9):
        bad = denoise.DnConfig(height=64, width=64, batch=1, levels=4, base_channels=32, in_channels=planes, seed=0)
        assert lib.dn_create(C.byref(bad), 0, C.byref(h)) == 1 and not h.value
    assert lib.dn_destroy(None) == 0
    assert lib.dn_conv2d_forward(None, 32, None, 0, 1, 8, 8, None, None, 3, 32, 1, None, 32, None) == 1
