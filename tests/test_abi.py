"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads, and
exports every entry point include/archer_epid.h declares; the ctypes struct
mirrors match the C layout.  No compute call is made (no GPU here)."""
import ctypes as C
import re
import subprocess
import textwrap
from pathlib import Path

import pytest

from paper_2510_24154_b300 import binding, build

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "archer_epid.h"


def declared_entry_points():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mc_[a-z_0-9]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert declared_entry_points() == sorted(binding.EXPORTED)


def test_library_builds_and_exports_every_symbol():
    lib_path = build.build()
    assert lib_path.exists()
    out = subprocess.run(["nm", "-D", "--defined-only", str(lib_path)], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(mc_\w+)", out))
    missing = set(declared_entry_points()) - exported
    assert not missing, f"missing exports: {missing}"
    lib = C.CDLL(str(lib_path))
    for name in declared_entry_points():
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


def test_struct_layouts_match_c(tmp_path):
    probe = textwrap.dedent("""
        #include <stdio.h>
        #include <stddef.h>
        #include "archer_epid.h"
        int main(void) {
          printf("%zu %zu %zu %zu %zu\\n", sizeof(mc_config), sizeof(mc_epid_desc), sizeof(mc_field_desc),
                 sizeof(mc_lut_desc), sizeof(mc_run_stats));
          printf("%zu %zu %zu %zu %zu %zu\\n", offsetof(mc_config, use_graph), offsetof(mc_config, regs_variant),
                 offsetof(mc_epid_desc, pitch_cm),
                 offsetof(mc_field_desc, eq1_literal), offsetof(mc_run_stats, gpu_ms),
                 offsetof(mc_run_stats, launches));
          return 0;
        }""")
    src = tmp_path / "probe.c"
    src.write_text(probe)
    exe = tmp_path / "probe"
    subprocess.run(["gcc", f"-I{ROOT / 'include'}", str(src), "-o", str(exe)], check=True)
    sizes, offs = [list(map(int, l.split())) for l in
                   subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()]
    assert sizes == [C.sizeof(binding.Config), C.sizeof(binding.EpidDesc), C.sizeof(binding.FieldDesc),
                     C.sizeof(binding.LutDesc), C.sizeof(binding.RunStats)]
    assert offs == [binding.Config.use_graph.offset, binding.Config.regs_variant.offset, binding.EpidDesc.pitch_cm.offset,
                    binding.FieldDesc.eq1_literal.offset, binding.RunStats.gpu_ms.offset,
                    binding.RunStats.launches.offset]
