"""Thin Python binding of libarcher_epid.so (the C ABI in include/archer_epid.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  There is no CPU fallback; if the library cannot be loaded, importing
this module raises.  Device buffers and streams come from PyTorch.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

from . import build as _build

MAX_LAYERS = 8
NUM_COUNTERS = 20
COUNTER_NAMES = ("flights_ct", "real_ct", "compton", "photo", "pair", "esteps_ct", "esteps_epid",
                 "moller", "brem", "primaries_at_epid", "uncollided_at_epid", "lost", "flights_epid",
                 "electrons", "positrons", "secondary_photons", "warp_iters_photon_ct", "live_lanes_photon_ct",
                 "warp_iters_electron_ct", "live_lanes_electron_ct")
STATUS = {0: "MC_OK", 1: "MC_ERR_ARG", 2: "MC_ERR_CUDA", 3: "MC_ERR_OOM", 4: "MC_ERR_STATE",
          5: "MC_ERR_TIMEOUT", 6: "MC_ERR_CANCELLED", 7: "MC_ERR_NUMERIC", 8: "MC_ERR_OVERFLOW"}

# Every entry point declared in include/archer_epid.h.
EXPORTED = ("mc_config_default", "mc_create", "mc_destroy", "mc_init_geometry", "mc_set_field", "mc_run",
            "mc_set_fields", "mc_run_batch", "mc_get_field_dose", "mc_get_field_image", "mc_get_field_tmap",
            "mc_get_field_size", "mc_get_dose", "mc_get_region_dose", "mc_get_field_fluence", "mc_get_epid_image", "mc_get_tmap", "mc_get_tally", "mc_field_size", "mc_get_stats",
            "mc_reset_tally", "mc_state_size", "mc_get_state", "mc_set_state", "mc_set_history_base", "mc_cancel",
            "mc_last_error",
            "mc_status_string", "mc_test_philox", "mc_test_uniforms", "mc_dose_stats_noalloc", "mc_gamma",
            "mc_get_patient_dose", "mc_get_plan_image", "mc_resample_image", "mc_probe_alu_peaks")


class Config(C.Structure):
    _fields_ = [("coupled", C.c_int), ("e_max_mev", C.c_double), ("mono_energy_mev", C.c_double),
                ("photon_cutoff_mev", C.c_double), ("electron_cutoff_mev", C.c_double),
                ("wcc_mev", C.c_double), ("wcb_mev", C.c_double), ("step_fraction", C.c_double),
                ("n_batches", C.c_int), ("max_steps", C.c_int), ("block_size", C.c_int),
                ("ctas_per_sm", C.c_int), ("bank_capacity", C.c_uint32), ("primaries_per_wave", C.c_uint32),
                ("time_kernels", C.c_int), ("use_graph", C.c_int), ("regs_variant", C.c_int * 4),
                ("patient_dose", C.c_int)]


class EpidDesc(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("material", C.c_int * MAX_LAYERS),
                ("thickness_cm", C.c_double * MAX_LAYERS), ("density", C.c_double * MAX_LAYERS),
                ("sensitive_layer", C.c_int), ("npx", C.c_int), ("npy", C.c_int), ("pitch_cm", C.c_double)]


class FieldDesc(C.Structure):
    _fields_ = [("n_segments", C.c_int), ("n_pairs", C.c_int), ("pair_edges_cm", C.POINTER(C.c_double)),
                ("leaves_cm", C.POINTER(C.c_double)), ("jaws_cm", C.POINTER(C.c_double)),
                ("mu", C.POINTER(C.c_double)), ("gantry_deg", C.c_double), ("sad_cm", C.c_double),
                ("sid_cm", C.c_double), ("iso_cm", C.c_double * 3), ("eq1_literal", C.c_int),
                ("leaf_transmission", C.c_double), ("jaw_transmission", C.c_double),
                ("tg_width_cm", C.c_double), ("leaf_gap_cm", C.c_double),
                ("leaf_thickness_cm", C.c_double), ("jaw_thickness_cm", C.c_double)]


class LutDesc(C.Structure):
    _fields_ = [("nt", C.c_int), ("ns", C.c_int), ("t_nodes", C.POINTER(C.c_double)),
                ("s_nodes", C.POINTER(C.c_double)), ("k", C.POINTER(C.c_double)), ("k_scale", C.c_double),
                ("t_offset_cm", C.c_double)]


class RunStats(C.Structure):
    _fields_ = [("histories", C.c_uint64), ("e_src_mev", C.c_double), ("e_ct_mev", C.c_double),
                ("e_epid_mev", C.c_double * MAX_LAYERS), ("e_esc_mev", C.c_double), ("e_lost_mev", C.c_double),
                ("counters", C.c_uint64 * NUM_COUNTERS), ("waves", C.c_int), ("error_flags", C.c_uint32),
                ("gpu_ms", C.c_double), ("kernel_ms", C.c_double * 4), ("kernel_launches", C.c_uint32 * 4),
                ("launches", C.c_uint32)]


class AluPeaks(C.Structure):
    _fields_ = [("ffma_tflops", C.c_double), ("ffma2_tflops", C.c_double), ("mufu_tops", C.c_double),
                ("int_tinst", C.c_double), ("mix_tinst", C.c_double), ("ms_total", C.c_double),
                ("sm_count", C.c_int32), ("_pad", C.c_int32)]


class MCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library_path() -> Path:
    return _build.LIB


def load(build_if_stale: bool = True):
    """Load (building first if the sources are newer) the CUDA library."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_stale:
        _build.build()
    if not _build.LIB.exists():
        raise ImportError(f"CUDA library {_build.LIB} is missing; run paper_2510_24154_b300/build.py")
    lib = C.CDLL(str(_build.LIB))
    P, vp, i, u64, u32, d = C.POINTER, C.c_void_p, C.c_int, C.c_uint64, C.c_uint32, C.c_double
    lib.mc_config_default.restype = None
    lib.mc_config_default.argtypes = [P(Config)]
    lib.mc_create.argtypes = [P(Config), i, P(vp)]
    lib.mc_destroy.argtypes = [vp]
    lib.mc_init_geometry.argtypes = [vp, vp, i, i, i, P(d), P(d), P(EpidDesc), i, vp]
    lib.mc_set_field.argtypes = [vp, P(FieldDesc), P(LutDesc), vp]
    lib.mc_run.argtypes = [vp, u64, u64, vp, P(RunStats)]
    lib.mc_set_fields.argtypes = [vp, P(FieldDesc), i, P(LutDesc), vp]
    lib.mc_run_batch.argtypes = [vp, P(u64), u64, vp, P(RunStats)]
    lib.mc_get_field_dose.argtypes = [vp, i, vp, vp, P(d), i, vp]
    lib.mc_get_field_image.argtypes = [vp, i, vp, i, vp]
    lib.mc_get_field_tmap.argtypes = [vp, i, vp, i, vp]
    lib.mc_get_field_size.argtypes = [vp, i, P(d), P(d), P(d)]
    lib.mc_get_dose.argtypes = [vp, vp, vp, P(d), i, vp]
    lib.mc_get_region_dose.argtypes = [vp, i, i, i, i, i, P(d), P(d), vp]
    lib.mc_get_field_fluence.argtypes = [vp, i, vp, i, vp]
    lib.mc_get_epid_image.argtypes = [vp, vp, i, vp]
    lib.mc_get_tmap.argtypes = [vp, vp, i, vp]
    lib.mc_get_tally.argtypes = [vp, vp, i, vp]
    lib.mc_field_size.argtypes = [vp, P(d), P(d), P(d)]
    lib.mc_get_stats.argtypes = [vp, P(RunStats)]
    lib.mc_reset_tally.argtypes = [vp, vp]
    lib.mc_state_size.argtypes = [vp, P(C.c_size_t)]
    lib.mc_get_state.argtypes = [vp, vp, C.c_size_t, vp]
    lib.mc_set_state.argtypes = [vp, vp, C.c_size_t, vp]
    lib.mc_cancel.argtypes = [vp]
    lib.mc_set_history_base.argtypes = [vp, u64]
    lib.mc_last_error.restype = C.c_char_p
    lib.mc_last_error.argtypes = [vp]
    lib.mc_status_string.restype = C.c_char_p
    lib.mc_status_string.argtypes = [i]
    lib.mc_test_philox.argtypes = [vp, vp, i, vp]
    lib.mc_test_uniforms.argtypes = [u64, u64, u32, i, vp, vp]
    lib.mc_dose_stats_noalloc.argtypes = [vp, i, i, i, u64, d, vp, vp, vp, vp]
    lib.mc_gamma.argtypes = [vp, vp, i, i, d, d, d, d, d, d, vp, P(d), vp]
    lib.mc_get_patient_dose.argtypes = [vp, vp, i, vp]
    lib.mc_get_plan_image.argtypes = [vp, vp, vp, vp, i, vp]
    lib.mc_resample_image.argtypes = [vp, i, i, d, vp, i, i, d, vp]
    lib.mc_probe_alu_peaks.argtypes = [i, i, P(AluPeaks)]
    for name in EXPORTED:
        if name not in ("mc_config_default", "mc_last_error", "mc_status_string"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def default_config(physics=None, **overrides) -> Config:
    lib = load()
    cfg = Config()
    lib.mc_config_default(C.byref(cfg))
    if physics is not None:
        cfg.coupled = int(physics.coupled)
        cfg.e_max_mev = physics.e_max
        cfg.mono_energy_mev = physics.mono_energy
        cfg.photon_cutoff_mev = physics.photon_cutoff
        cfg.electron_cutoff_mev = physics.electron_cutoff
        cfg.wcc_mev = physics.wcc
        cfg.wcb_mev = physics.wcb
        cfg.step_fraction = physics.step_fraction
        cfg.n_batches = physics.n_batches
        cfg.max_steps = physics.max_steps
    for k, v in overrides.items():
        if k == "regs_variant":
            cfg.regs_variant[:] = list(v)
        else:
            setattr(cfg, k, v)
    return cfg


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(x):
    """Device pointer of a torch tensor, or host pointer of a numpy array."""
    if isinstance(x, np.ndarray):
        return C.c_void_p(x.ctypes.data)
    return C.c_void_p(x.data_ptr())


class Simulator:
    """One library context on one GPU: geometry, field, runs and read-outs."""

    def __init__(self, physics=None, device: int = 0, **overrides):
        self.lib = load()
        self.cfg = default_config(physics, **overrides)
        h = C.c_void_p()
        self._check(self.lib.mc_create(C.byref(self.cfg), device, C.byref(h)), None)
        self.h = h
        self.device = device
        self.epid = None
        self.n_fields = 0
        self._keep = []

    def _check(self, st, h="self"):
        if st != 0:
            hh = self.h if h == "self" else h
            msg = self.lib.mc_last_error(hh).decode() if hh else self.lib.mc_status_string(st).decode()
            raise MCError(st, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.mc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up -------------------------------------------------------------
    def init_geometry(self, phantom, epid, stream=None, hu_device=None):
        """CT set-up (Sec. 2.1.2): HU volume (numpy int16 [nz][ny][nx], or a CUDA int16 tensor via hu_device)."""
        nz, ny, nx = phantom.hu.shape
        vox = (C.c_double * 3)(*phantom.vox)
        org = (C.c_double * 3)(*phantom.origin)
        e = EpidDesc()
        e.n_layers = len(epid.layers)
        for l, (m, t, r) in enumerate(epid.layers):
            e.material[l], e.thickness_cm[l], e.density[l] = int(m), float(t), float(r)
        e.sensitive_layer, e.npx, e.npy, e.pitch_cm = epid.sensitive, epid.npx, epid.npy, epid.pitch
        if hu_device is not None:
            ptr, on_dev = _ptr(hu_device), 1
        else:
            hu = np.ascontiguousarray(phantom.hu, dtype=np.int16)
            self._keep = [hu]
            ptr, on_dev = C.c_void_p(hu.ctypes.data), 0
        self._check(self.lib.mc_init_geometry(self.h, ptr, nx, ny, nz, vox, org, C.byref(e), on_dev,
                                              _stream_ptr(stream)))
        self.epid = epid
        self._ct_shape = (nz, ny, nx)

    @staticmethod
    def _field_desc(field, lut, keep):
        edges = np.ascontiguousarray(field.pair_edges, dtype=np.float64)
        leaves = np.ascontiguousarray(field.leaves, dtype=np.float64)
        jaws = np.ascontiguousarray(field.jaws, dtype=np.float64)
        mu = np.ascontiguousarray(field.mu, dtype=np.float64)
        keep += [edges, leaves, jaws, mu]
        f = FieldDesc()
        f.n_segments, f.n_pairs = leaves.shape[0], leaves.shape[1]
        f.pair_edges_cm, f.leaves_cm, f.jaws_cm, f.mu = _dp(edges), _dp(leaves), _dp(jaws), _dp(mu)
        f.gantry_deg, f.sad_cm, f.sid_cm = field.gantry_deg, field.sad, field.sid
        f.iso_cm[:] = [float(v) for v in field.iso]
        f.eq1_literal = int(lut.eq1_literal) if lut is not None else 0
        f.leaf_transmission = float(getattr(field, "leaf_transmission", 0.0))
        f.jaw_transmission = float(getattr(field, "jaw_transmission", 0.0))
        f.tg_width_cm = float(getattr(field, "tg_width", 0.0))
        f.leaf_gap_cm = float(getattr(field, "leaf_gap", 0.0))
        f.leaf_thickness_cm = float(getattr(field, "leaf_thickness", 0.0))
        f.jaw_thickness_cm = float(getattr(field, "jaw_thickness", 0.0))
        return f

    @staticmethod
    def _lut_desc(lut, keep):
        if lut is None:
            return None
        tn = np.ascontiguousarray(lut.t_nodes, dtype=np.float64)
        sn = np.ascontiguousarray(lut.s_nodes, dtype=np.float64)
        k = np.ascontiguousarray(lut.k, dtype=np.float64)
        keep += [tn, sn, k]
        L = LutDesc()
        L.nt, L.ns = tn.size, sn.size
        L.t_nodes, L.s_nodes, L.k = _dp(tn), _dp(sn), _dp(k)
        L.k_scale, L.t_offset_cm = lut.k_scale, lut.t_offset
        keep.append(L)
        return C.byref(L)

    def set_field(self, field, lut=None, stream=None):
        """Source set-up (Sec. 2.1.1), t-map (Sec. 2.2), Eq. 1, k-table upload; resets the tally."""
        keep = []
        f = self._field_desc(field, lut, keep)
        lp = self._lut_desc(lut, keep)
        self._check(self.lib.mc_set_field(self.h, C.byref(f), lp, _stream_ptr(stream)))
        self.n_fields = 1

    def set_fields(self, fields, lut=None, stream=None):
        """Several fields of one plan (own source, gantry angle, t-map, s and tally each)."""
        keep = []
        arr = (FieldDesc * len(fields))(*[self._field_desc(f, lut, keep) for f in fields])
        lp = self._lut_desc(lut, keep)
        self._check(self.lib.mc_set_fields(self.h, arr, len(fields), lp, _stream_ptr(stream)))
        self.n_fields = len(fields)

    # -- transport ------------------------------------------------------------
    def run(self, n_histories, seed, stream=None) -> dict:
        """Transport (Sec. 2.1) of n_histories more histories; waits and returns the stats."""
        st = RunStats()
        self._check(self.lib.mc_run(self.h, int(n_histories), int(seed), _stream_ptr(stream), C.byref(st)))
        return stats_dict(st)

    def run_async(self, n_histories, seed, stream=None) -> None:
        """Transport (Sec. 2.1) queued on `stream` (graph-driven runs return at once); the
        stats and any device-side failure come from stats()."""
        self._check(self.lib.mc_run(self.h, int(n_histories), int(seed), _stream_ptr(stream), None))

    def run_batch(self, n_histories, seed, stream=None) -> dict:
        """n_histories[f] more histories of every field f, in one wave sequence."""
        n = (C.c_uint64 * self.n_fields)(*[int(v) for v in n_histories])
        st = RunStats()
        self._check(self.lib.mc_run_batch(self.h, n, int(seed), _stream_ptr(stream), C.byref(st)))
        return stats_dict(st)

    def stats(self) -> dict:
        st = RunStats()
        self._check(self.lib.mc_get_stats(self.h, C.byref(st)))
        return stats_dict(st)

    # -- read-outs ------------------------------------------------------------
    def _npix(self):
        return self.epid.npy, self.epid.npx

    def dose(self, stream=None, with_sigma=True, field=0):
        """Dose statistics (Sec. 2.3): (dose, sigma, u) as numpy arrays (Gy per history) and the scalar u."""
        ny, nx = self._npix()
        d = np.empty((ny, nx))
        s = np.empty((ny, nx)) if with_sigma else None
        u = C.c_double()
        self._check(self.lib.mc_get_field_dose(self.h, int(field), C.c_void_p(d.ctypes.data),
                                               C.c_void_p(s.ctypes.data) if s is not None else None,
                                               C.byref(u) if with_sigma else None, 0, _stream_ptr(stream)))
        return d, s, u.value

    def dose_device(self, dose, sigma=None, stream=None, field=0):
        self._check(self.lib.mc_get_field_dose(self.h, int(field), _ptr(dose),
                                               _ptr(sigma) if sigma is not None else None, None, 1,
                                               _stream_ptr(stream)))

    def fluence(self, stream=None, field=0):
        """Source fluence density (cm^-2 at the isocentre plane) at the EPID
        pixel centres, float64 numpy [npy][npx]."""
        ny, nx = self._npix()
        out = np.empty((ny, nx))
        self._check(self.lib.mc_get_field_fluence(self.h, int(field), C.c_void_p(out.ctypes.data), 0,
                                                  _stream_ptr(stream)))
        return out

    def fluence_device(self, out, stream=None, field=0):
        """As fluence(), into a CUDA float64 tensor [npy][npx] (queued on the stream)."""
        self._check(self.lib.mc_get_field_fluence(self.h, int(field), _ptr(out), 1, _stream_ptr(stream)))

    def tmap_device(self, out, stream=None, field=0):
        """The t-map into a CUDA float64 tensor [npy][npx] (queued on the stream)."""
        self._check(self.lib.mc_get_field_tmap(self.h, int(field), _ptr(out), 1, _stream_ptr(stream)))

    def region_dose(self, ix0, ix1, iy0, iy1, stream=None, field=0):
        """Mean per-history dose (Gy) over pixels [ix0, ix1) x [iy0, iy1) and
        the batch standard error of that mean, computed on the device."""
        m, e = C.c_double(), C.c_double()
        self._check(self.lib.mc_get_region_dose(self.h, int(field), int(ix0), int(ix1), int(iy0), int(iy1),
                                                C.byref(m), C.byref(e), _stream_ptr(stream)))
        return m.value, e.value

    def epid_image(self, stream=None, field=0):
        """The k(t, s)-corrected signal (Sec. 3.1), float32 numpy [npy][npx]."""
        ny, nx = self._npix()
        out = np.empty((ny, nx), dtype=np.float32)
        self._check(self.lib.mc_get_field_image(self.h, int(field), C.c_void_p(out.ctypes.data), 0,
                                                _stream_ptr(stream)))
        return out

    def epid_image_device(self, out, stream=None, field=0):
        self._check(self.lib.mc_get_field_image(self.h, int(field), _ptr(out), 1, _stream_ptr(stream)))

    def tmap(self, stream=None, field=0):
        ny, nx = self._npix()
        out = np.empty((ny, nx))
        self._check(self.lib.mc_get_field_tmap(self.h, int(field), C.c_void_p(out.ctypes.data), 0,
                                               _stream_ptr(stream)))
        return out

    def tally_all(self, stream=None):
        """Raw sub-tallies of every field, uint64 [n_fields][B][npy][npx] (unit 2^-8 eV)."""
        ny, nx = self._npix()
        out = np.empty((self.n_fields, self.cfg.n_batches, ny, nx), dtype=np.uint64)
        self._check(self.lib.mc_get_tally(self.h, C.c_void_p(out.ctypes.data), 0, _stream_ptr(stream)))
        return out

    def tally(self, stream=None, field=0):
        """Raw sub-tallies of one field, uint64 [B][npy][npx]."""
        return self.tally_all(stream)[field]

    def plan_image(self, weights=None, stream=None):
        """Weighted sums over the fields: (dose, signal) [npy][npx] (signal None without a k-table)."""
        ny, nx = self._npix()
        d = np.empty((ny, nx))
        sg = np.empty((ny, nx))
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
        self._check(self.lib.mc_get_plan_image(self.h, C.c_void_p(w.ctypes.data) if w is not None else None,
                                               C.c_void_p(d.ctypes.data), C.c_void_p(sg.ctypes.data), 0,
                                               _stream_ptr(stream)))
        return d, sg

    def patient_dose(self, stream=None):
        """Per-history dose (Gy) of every CT voxel [nz][ny][nx] (needs patient_dose=1)."""
        nz, ny, nx = self._ct_shape
        out = np.empty((nz, ny, nx))
        self._check(self.lib.mc_get_patient_dose(self.h, C.c_void_p(out.ctypes.data), 0, _stream_ptr(stream)))
        return out

    def field_size(self, field=0):
        s, a, b = C.c_double(), C.c_double(), C.c_double()
        self._check(self.lib.mc_get_field_size(self.h, int(field), C.byref(s), C.byref(a), C.byref(b)))
        return s.value, a.value, b.value

    def set_history_base(self, next_history):
        self._check(self.lib.mc_set_history_base(self.h, int(next_history)))

    def reset_tally(self, stream=None):
        self._check(self.lib.mc_reset_tally(self.h, _stream_ptr(stream)))

    def get_state(self, stream=None) -> bytes:
        n = C.c_size_t()
        self._check(self.lib.mc_state_size(self.h, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(self.lib.mc_get_state(self.h, buf, n.value, _stream_ptr(stream)))
        return bytes(buf.raw)

    def set_state(self, blob: bytes, stream=None):
        buf = C.create_string_buffer(blob, len(blob))
        self._check(self.lib.mc_set_state(self.h, buf, len(blob), _stream_ptr(stream)))


def stats_dict(st: RunStats) -> dict:
    return {
        "histories": int(st.histories),
        "e_src": st.e_src_mev, "e_ct": st.e_ct_mev, "e_epid": np.array(st.e_epid_mev[:]),
        "e_esc": st.e_esc_mev, "e_lost": st.e_lost_mev,
        "counters": dict(zip(COUNTER_NAMES, [int(v) for v in st.counters])),
        "waves": int(st.waves), "error_flags": int(st.error_flags), "gpu_ms": float(st.gpu_ms),
        "kernel_ms": [float(v) for v in st.kernel_ms], "kernel_launches": [int(v) for v in st.kernel_launches],
        "launches": int(st.launches),
    }


def test_philox(ctr_key, stream=None):
    """Philox4x32-10 on the GPU for rows (ctr0..3, key0, key1); returns [n][4] uint32."""
    import torch
    lib = load()
    a = torch.as_tensor(np.ascontiguousarray(ctr_key, dtype=np.uint32).view(np.int32), device="cuda")
    out = torch.empty((a.shape[0], 4), dtype=torch.int32, device="cuda")
    st = lib.mc_test_philox(_ptr(a), _ptr(out), a.shape[0], _stream_ptr(stream))
    if st:
        raise MCError(st, "mc_test_philox")
    return out.cpu().numpy().view(np.uint32)


def test_uniforms(seed, hist, ord_, n, stream=None):
    import torch
    lib = load()
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    st = lib.mc_test_uniforms(int(seed), int(hist), int(ord_), int(n), _ptr(out), _stream_ptr(stream))
    if st:
        raise MCError(st, "mc_test_uniforms")
    return out.cpu().numpy()


def probe_alu_peaks(device=0, repeats=3):
    """mc_probe_alu_peaks: measured FP32 FMA (scalar and f32x2), ex2/lg2,
    integer and mixed-issue rates of the GPU, as a dict."""
    lib = load()
    r = AluPeaks()
    st = lib.mc_probe_alu_peaks(int(device), int(repeats), C.byref(r))
    if st:
        raise MCError(st, "mc_probe_alu_peaks")
    return {k: getattr(r, k) for k, _ in AluPeaks._fields_ if not k.startswith("_")}


def dose_stats_noalloc(tally, npx, npy, n_batches, n_histories, pixel_mass_kg, dose, sigma=None, u=None,
                       stream=None):
    """mc_dose_stats_noalloc on device tensors (tally int64 [B][npy][npx],
    dose/sigma float64 [npy][npx], u float64 [1]); allocates nothing."""
    lib = load()
    st = lib.mc_dose_stats_noalloc(_ptr(tally), int(npx), int(npy), int(n_batches), int(n_histories),
                                   float(pixel_mass_kg), _ptr(dose), _ptr(sigma) if sigma is not None else None,
                                   _ptr(u) if u is not None else None, _stream_ptr(stream))
    if st:
        raise MCError(st, "mc_dose_stats_noalloc")


def gamma(ref, ev, pixel_mm, dd=0.01, dta_mm=1.0, threshold=0.10, step_mm=0.0, radius_mm=0.0, out=None,
          stream=None):
    """Global gamma pass rate of `ev` against `ref` (CUDA float64 tensors
    [ny][nx]); per-pixel values go to `out` (same shape) when given."""
    lib = load()
    ny, nx = ref.shape
    rate = C.c_double()
    st = lib.mc_gamma(_ptr(ref), _ptr(ev), nx, ny, float(pixel_mm), float(dd), float(dta_mm), float(threshold),
                      float(step_mm), float(radius_mm), _ptr(out) if out is not None else None, C.byref(rate),
                      _stream_ptr(stream))
    if st != 0:
        raise MCError(st, "mc_gamma failed")
    return rate.value


def resample_image(src, src_pitch, dst, dst_pitch, stream=None):
    """Bilinear resampling of a CUDA float64 image onto `dst`'s grid (same centre)."""
    lib = load()
    sny, snx = src.shape
    dny, dnx = dst.shape
    st = lib.mc_resample_image(_ptr(src), snx, sny, float(src_pitch), _ptr(dst), dnx, dny, float(dst_pitch),
                               _stream_ptr(stream))
    if st != 0:
        raise MCError(st, "mc_resample_image failed")
