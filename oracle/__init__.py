"""FP64 CPU oracle for the EPID transit Monte Carlo path.

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py`` (``cpu_baseline`` and ``--impl reference``).  The
CUDA product path never imports it.  It shares no code with the CUDA library:
transport, ray tracing and gamma live in ``archer_oracle.c`` (plain C, double
precision, built with gcc), and the short closed-form steps below (Eq. 1, the
bilinear k(t,s) lookup of Sec. 3.1, batch statistics) are plain numpy in FP64.

Pins: every function here is checked in ``tests/test_oracle_*.py`` against
something other than itself (closed forms, numerical integration, brute-force
enumeration, the paper's Table 1).  The magnitudes of the builder's
photoelectric, pair and bremsstrahlung fits have no external data to compare
with in this container: parity unpinned for those magnitudes, while their
structure (exponents, edge, threshold, mixture rule) is pinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "archer_oracle.c"
_LIB = _HERE / "liborc.so"

MAXL = 8
COUNTER_NAMES = ("flights_ct", "real_ct", "compton", "photo", "pair", "esteps_ct", "esteps_epid",
                 "moller", "brem", "primaries_at_epid", "uncollided_at_epid", "lost", "flights_epid",
                 "electrons", "positrons", "secondary_photons")


def build(force: bool = False) -> Path:
    """Compile the C oracle with gcc (a plain -O2 build, no fast-math)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".{os.getpid()}.tmp.so")
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", str(tmp), str(_SRC),
                        "-lm", "-lpthread"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("hu", C.POINTER(C.c_int16)), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("vox", C.c_double * 3), ("origin", C.c_double * 3),
        ("n_layers", C.c_int), ("layer_mat", C.c_int * MAXL), ("layer_thick", C.c_double * MAXL),
        ("layer_rho", C.c_double * MAXL), ("sens_layer", C.c_int), ("npx", C.c_int), ("npy", C.c_int),
        ("pitch", C.c_double),
        ("n_seg", C.c_int), ("n_pairs", C.c_int), ("pair_edges", C.POINTER(C.c_double)),
        ("leaves", C.POINTER(C.c_double)), ("jaws", C.POINTER(C.c_double)), ("mu", C.POINTER(C.c_double)),
        ("gantry_deg", C.c_double), ("sad", C.c_double), ("sid", C.c_double), ("iso", C.c_double * 3),
        ("coupled", C.c_int), ("e_max", C.c_double), ("mono_e", C.c_double), ("pcut", C.c_double),
        ("ecut", C.c_double), ("wcc", C.c_double), ("wcb", C.c_double), ("step_frac", C.c_double),
        ("n_batches", C.c_int), ("max_steps", C.c_int), ("leaf_trans", C.c_double),
        ("jaw_trans", C.c_double), ("tg_width", C.c_double), ("leaf_gap", C.c_double),
        ("leaf_thick", C.c_double), ("jaw_thick", C.c_double),
    ]


class _Result(C.Structure):
    _fields_ = [
        ("tally", C.POINTER(C.c_double)), ("e_src", C.c_double), ("e_ct", C.c_double),
        ("e_epid", C.c_double * MAXL), ("e_esc", C.c_double), ("e_lost", C.c_double),
        ("counters", C.c_uint64 * len(COUNTER_NAMES)), ("vox", C.POINTER(C.c_double)),
    ]


class _Probe(C.Structure):
    _fields_ = [
        ("type", C.c_int), ("E", C.c_double), ("x", C.c_double * 3), ("u", C.c_double * 3),
        ("no_ms", C.c_int), ("no_hard", C.c_int), ("macro_M", C.c_int), ("cap", C.c_int64),
        ("path", C.POINTER(C.c_double)), ("hard_T", C.POINTER(C.c_double)), ("hard_type", C.POINTER(C.c_int32)),
        ("first_layer", C.POINTER(C.c_int32)), ("first_pos", C.POINTER(C.c_double)),
        ("end_pos", C.POINTER(C.c_double)), ("first_pixel", C.POINTER(C.c_int64)),
        ("pair_frac", C.POINTER(C.c_double)), ("annih_cos", C.POINTER(C.c_double)),
        ("annih_phi", C.POINTER(C.c_double)), ("brem_x", C.POINTER(C.c_double)),
        ("compton_phi", C.POINTER(C.c_double)),
        ("n_exit_uncollided", C.c_uint64), ("n_compton", C.c_uint64), ("n_moller", C.c_uint64),
        ("n_brem", C.c_uint64), ("n_pair", C.c_uint64), ("n_annih", C.c_uint64), ("n_pos_escape", C.c_uint64),
        ("n_pos_born", C.c_uint64),
        ("compton_dev", C.c_double), ("polar_dev", C.c_double), ("moller_dev", C.c_double),
        ("brem_dev", C.c_double),
        ("pair_dev", C.c_double), ("annih_dev", C.c_double), ("unit_dev", C.c_double),
        ("hidx", C.c_int64), ("first_done", C.c_int), ("pix_done", C.c_int), ("hard_done", C.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(str(build()))
        d, i, u64, u32 = C.c_double, C.c_int, C.c_uint64, C.c_uint32
        P = C.POINTER
        _lib.orc_sigma_kn.restype = d
        _lib.orc_sigma_kn.argtypes = [d]
        _lib.orc_mu_photon.argtypes = [i, d, P(d)]
        for name in ("orc_lcol", "orc_sigma_moller", "orc_lrad_soft", "orc_sigma_brem"):
            getattr(_lib, name).restype = d
            getattr(_lib, name).argtypes = [i, d, d]
        _lib.orc_lambda1_inv.restype = d
        _lib.orc_lambda1_inv.argtypes = [i, d]
        _lib.orc_wentzel_A.restype = d
        _lib.orc_wentzel_A.argtypes = [d]
        _lib.orc_philox.argtypes = [P(u32), P(u32), P(u32)]
        _lib.orc_child_ordinal.restype = u32
        _lib.orc_child_ordinal.argtypes = [u32, u32, u32]
        _lib.orc_uniforms.argtypes = [u64, u64, u32, u32, P(d)]
        _lib.orc_sample_kn_many.argtypes = [d, u64, u64, P(d), P(d)]
        _lib.orc_sample_spectrum_many.argtypes = [d, d, u64, u64, P(d)]
        _lib.orc_sample_moller_many.argtypes = [d, d, u64, u64, P(d)]
        _lib.orc_sample_ms_many.argtypes = [d, u64, u64, P(d)]
        _lib.orc_csda_path.restype = d
        _lib.orc_csda_path.argtypes = [i, d, d, d, d, d, d]
        _lib.orc_hu_to_rho_mat.argtypes = [i, P(d), P(i)]
        _lib.orc_run.restype = i
        _lib.orc_run.argtypes = [P(_Problem), u64, u64, u64, i, P(_Result)]
        _lib.orc_first_interaction.argtypes = [P(_Problem), d, P(d), P(d), u64, u64, i, P(C.c_int64),
                                               P(C.c_int32)]
        _lib.orc_pencil.restype = i
        _lib.orc_pencil.argtypes = [P(_Problem), P(_Probe), u64, u64, u64, P(_Result)]
        _lib.orc_tmap.argtypes = [P(_Problem), P(C.c_int32), P(C.c_int32), C.c_int64, P(d)]
        _lib.orc_siddon_ray.restype = d
        _lib.orc_siddon_ray.argtypes = [P(_Problem), P(d), P(d)]
        _lib.orc_sample_ps2_many.restype = i
        _lib.orc_sample_ps2_many.argtypes = [P(_Problem), u64, u64, u64, P(d), P(d), P(d), P(C.c_int32),
                                             P(C.c_int32)]
        _lib.orc_sample_source_many.restype = i
        _lib.orc_sample_source_many.argtypes = [P(_Problem), u64, u64, u64, P(d), P(d), P(d)]
        _lib.orc_gamma.restype = d
        _lib.orc_gamma.argtypes = [P(d), P(d), i, i, d, d, d, d, d, d, P(d)]
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _Marshalled:
    """Keeps the numpy buffers alive while the C struct points at them."""

    def __init__(self, problem, physics=None, field=None):
        ph, ep = problem.phantom, problem.epid
        fld = field if field is not None else problem.field
        phy = physics if physics is not None else problem.physics
        self.hu = np.ascontiguousarray(ph.hu, dtype=np.int16)
        self.edges = np.ascontiguousarray(fld.pair_edges, dtype=np.float64)
        self.leaves = np.ascontiguousarray(fld.leaves, dtype=np.float64)
        self.jaws = np.ascontiguousarray(fld.jaws, dtype=np.float64)
        self.mu = np.ascontiguousarray(fld.mu, dtype=np.float64)
        s = _Problem()
        s.hu = self.hu.ctypes.data_as(C.POINTER(C.c_int16))
        nz, ny, nx = self.hu.shape
        s.nx, s.ny, s.nz = nx, ny, nz
        s.vox[:] = [float(v) for v in ph.vox]
        s.origin[:] = [float(v) for v in ph.origin]
        if not 1 <= len(ep.layers) <= MAXL:
            raise ValueError("EPID needs 1..8 layers")
        s.n_layers = len(ep.layers)
        for l, (m, t, r) in enumerate(ep.layers):
            s.layer_mat[l], s.layer_thick[l], s.layer_rho[l] = int(m), float(t), float(r)
        s.sens_layer, s.npx, s.npy, s.pitch = ep.sensitive, ep.npx, ep.npy, ep.pitch
        s.n_seg, s.n_pairs = self.leaves.shape[0], self.leaves.shape[1]
        s.pair_edges, s.leaves, s.jaws, s.mu = _dp(self.edges), _dp(self.leaves), _dp(self.jaws), _dp(self.mu)
        s.gantry_deg, s.sad, s.sid = fld.gantry_deg, fld.sad, fld.sid
        s.iso[:] = [float(v) for v in fld.iso]
        s.coupled = int(phy.coupled)
        s.e_max, s.mono_e = phy.e_max, phy.mono_energy
        s.pcut, s.ecut, s.wcc, s.wcb = phy.photon_cutoff, phy.electron_cutoff, phy.wcc, phy.wcb
        s.step_frac, s.n_batches, s.max_steps = phy.step_fraction, phy.n_batches, phy.max_steps
        s.leaf_trans = float(getattr(fld, "leaf_transmission", 0.0))
        s.jaw_trans = float(getattr(fld, "jaw_transmission", 0.0))
        s.tg_width = float(getattr(fld, "tg_width", 0.0))
        s.leaf_gap = float(getattr(fld, "leaf_gap", 0.0))
        s.leaf_thick = float(getattr(fld, "leaf_thickness", 0.0))
        s.jaw_thick = float(getattr(fld, "jaw_thickness", 0.0))
        if not (0.0 <= s.leaf_thick <= 20.0 and 0.0 <= s.jaw_thick < 23.0):
            raise ValueError("need 0 <= leaf slab <= 20 cm and 0 <= jaw slab < 23 cm")
        if (s.leaf_thick > 0.0 or s.jaw_thick > 0.0) and (s.leaf_trans > 0.0 or s.jaw_trans > 0.0):
            raise ValueError("collimator slabs replace the transmission factors: set those to 0")
        edges = np.asarray(fld.pair_edges, dtype=np.float64)
        if not (0.0 <= s.leaf_trans < 1.0 and 0.0 <= s.jaw_trans < 1.0):
            raise ValueError("transmissions must lie in [0, 1)")
        if not (0.0 <= s.tg_width < np.diff(edges).min()) or not (0.0 <= s.leaf_gap < 2.0):
            raise ValueError("need 0 <= tongue-and-groove width < narrowest pair and 0 <= leaf gap < 2 cm")
        self.s = s


def run(problem, n_histories=None, seed=None, hist_begin=0, threads=None, physics=None, field=None,
        patient_dose=False):
    """Transport `n_histories` histories (ids hist_begin..) and return the tally
    [B][npy][npx] in MeV, the energy balance and the event counters; with
    patient_dose, also "vox": the energy (MeV) deposited in each CT voxel,
    [nz][ny][nx]."""
    m = _Marshalled(problem, physics, field)
    n = int(problem.n_histories if n_histories is None else n_histories)
    sd = int(problem.seed if seed is None else seed)
    B = m.s.n_batches
    tally = np.zeros((B, m.s.npy, m.s.npx), dtype=np.float64)
    r = _Result()
    r.tally = _dp(tally)
    vox = np.zeros(problem.phantom.hu.shape, dtype=np.float64) if patient_dose else None
    if vox is not None:
        r.vox = _dp(vox)
    nthr = int(threads if threads is not None else (os.cpu_count() or 1))
    rc = lib().orc_run(C.byref(m.s), sd, int(hist_begin), n, nthr, C.byref(r))
    if rc != 0:
        raise RuntimeError(f"orc_run failed with code {rc}")
    return {
        "tally": tally,
        "e_src": r.e_src, "e_ct": r.e_ct, "e_epid": np.array(r.e_epid[:len(problem.epid.layers)]),
        "e_esc": r.e_esc, "e_lost": r.e_lost,
        "counters": dict(zip(COUNTER_NAMES, [int(v) for v in r.counters])),
        "threads": min(nthr, B), "vox": vox,
    }


def first_interaction(problem, E, start, direction, n, seed=0, macro_M=0):
    """First real interaction (flat voxel, type) of n photons along one ray;
    macro_M > 0 overrides the macro-cell size of the Woodcock majorant."""
    m = _Marshalled(problem)
    st = np.ascontiguousarray(start, dtype=np.float64)
    dr = np.ascontiguousarray(direction, dtype=np.float64)
    vox = np.empty(n, dtype=np.int64)
    typ = np.empty(n, dtype=np.int32)
    lib().orc_first_interaction(C.byref(m.s), float(E), _dp(st), _dp(dr), int(seed), int(n), int(macro_M),
                                vox.ctypes.data_as(C.POINTER(C.c_int64)),
                                typ.ctypes.data_as(C.POINTER(C.c_int32)))
    return vox, typ


PARTICLE = {"photon": 0, "electron": 1, "positron": 2}
_PROBE_SAMPLES = ("pair_frac", "annih_cos", "annih_phi", "brem_x", "compton_phi")
_PROBE_COUNTS = ("n_exit_uncollided", "n_compton", "n_moller", "n_brem", "n_pair", "n_annih", "n_pos_escape",
                 "n_pos_born")
_PROBE_DEVS = ("compton_dev", "polar_dev", "moller_dev", "brem_dev", "pair_dev", "annih_dev", "unit_dev")


def pencil(problem, particle, E, start, direction, n, seed=0, hist_begin=0, no_ms=False, no_hard=False,
           macro_M=0, patient_dose=False, cap=200_000, threads=None, physics=None, field=None):
    """Histories whose primary is one given particle (a pencil), transported
    by the oracle's own transport with its test probe recording (orc_pencil).

    particle: "photon", "electron" or "positron"; start/direction in the
    patient frame (a charged primary starts inside the CT; a photon enters
    the world along its line).  no_ms / no_hard switch off the deflections /
    the hard events.  Returns the usual energy balance, tally and counters
    plus, per history, "path" (charged primary's track length), "hard_T" /
    "hard_type" (its first hard event), "first_layer", "first_pos" and
    "first_pixel" (a photon primary's first real interaction and first
    deposit), "end_pos" (where a charged primary stops), the kinematic deviations, event counts and up to `cap` samples
    per thread of each kind.  Chunks of histories run on `threads` threads
    (the C call releases the GIL); each history is independent."""
    from concurrent.futures import ThreadPoolExecutor
    m = _Marshalled(problem, physics, field)
    n = int(n)
    nthr = max(1, min(int(threads if threads is not None else (os.cpu_count() or 1)), n))
    B = m.s.n_batches
    bounds = np.linspace(0, n, nthr + 1).astype(np.int64)
    out = {"path": np.zeros(n), "hard_T": np.zeros(n), "hard_type": np.zeros(n, np.int32),
           "first_layer": np.zeros(n, np.int32), "first_pos": np.zeros((n, 3)), "end_pos": np.zeros((n, 3)),
           "first_pixel": np.zeros(n, np.int64)}
    st = np.ascontiguousarray(start, dtype=np.float64)
    dr = np.ascontiguousarray(direction, dtype=np.float64)

    def chunk(k):
        a, b = int(bounds[k]), int(bounds[k + 1])
        q = _Probe()
        q.type, q.E = PARTICLE[particle], float(E)
        q.x[:], q.u[:] = [float(v) for v in st], [float(v) for v in dr]
        q.no_ms, q.no_hard, q.macro_M, q.cap = int(no_ms), int(no_hard), int(macro_M), int(cap)
        views = {key: arr[a:b] for key, arr in out.items()}
        keep = [views]
        q.path, q.hard_T = _dp(views["path"]), _dp(views["hard_T"])
        q.hard_type = views["hard_type"].ctypes.data_as(C.POINTER(C.c_int32))
        q.first_layer = views["first_layer"].ctypes.data_as(C.POINTER(C.c_int32))
        q.first_pos = _dp(views["first_pos"])
        q.end_pos = _dp(views["end_pos"])
        q.first_pixel = views["first_pixel"].ctypes.data_as(C.POINTER(C.c_int64))
        samples = {key: np.full(int(cap), np.nan) for key in _PROBE_SAMPLES}
        for key, arr in samples.items():
            setattr(q, key, _dp(arr))
        tally = np.zeros((B, m.s.npy, m.s.npx), dtype=np.float64)
        r = _Result()
        r.tally = _dp(tally)
        vox = np.zeros(problem.phantom.hu.shape, dtype=np.float64) if patient_dose else None
        if vox is not None:
            r.vox = _dp(vox)
        rc = lib().orc_pencil(C.byref(m.s), C.byref(q), int(seed), int(hist_begin) + a, b - a, C.byref(r))
        if rc != 0:
            raise RuntimeError(f"orc_pencil failed with code {rc}")
        del keep
        return q, r, tally, vox, samples

    with ThreadPoolExecutor(nthr) as ex:
        parts = list(ex.map(chunk, range(nthr)))
    res = dict(out)
    res["tally"] = sum(p[2] for p in parts)
    res["vox"] = sum(p[3] for p in parts) if patient_dose else None
    res["e_src"] = sum(p[1].e_src for p in parts)
    res["e_ct"] = sum(p[1].e_ct for p in parts)
    res["e_esc"] = sum(p[1].e_esc for p in parts)
    res["e_lost"] = sum(p[1].e_lost for p in parts)
    res["e_epid"] = sum(np.array(p[1].e_epid[:len(problem.epid.layers)]) for p in parts)
    res["counters"] = {name: sum(int(p[1].counters[i]) for p in parts) for i, name in enumerate(COUNTER_NAMES)}
    for key in _PROBE_COUNTS:
        res[key] = sum(int(getattr(p[0], key)) for p in parts)
    for key in _PROBE_DEVS:
        res[key] = max(float(getattr(p[0], key)) for p in parts)
    for key in _PROBE_SAMPLES:
        vals = [p[4][key] for p in parts]
        cnt = {"pair_frac": "n_pair", "annih_cos": "n_annih", "annih_phi": "n_annih", "brem_x": "n_brem",
               "compton_phi": "n_compton"}[key]
        res[key] = np.concatenate([v[:min(int(getattr(p[0], cnt)), int(cap))] for v, p in zip(vals, parts)])
    return res


def sample_source(problem, n, seed=0, hist_begin=0):
    """Isocentre-plane points (X, Y) and energies of the primaries of histories
    hist_begin.. drawn exactly as the transport draws them."""
    m = _Marshalled(problem)
    X, Y, E = np.empty(n), np.empty(n), np.empty(n)
    rc = lib().orc_sample_source_many(C.byref(m.s), int(seed), int(hist_begin), int(n), _dp(X), _dp(Y), _dp(E))
    if rc:
        raise RuntimeError("field has no open aperture")
    return X, Y, E


def sample_ps2(problem, n, seed=0, hist_begin=0, physics=None, field=None):
    """Phase-space-2 photons of histories hist_begin.. as the transport draws
    them (collimator slabs crossed): the source ray's isocentre-plane point
    (X, Y), the energy (NaN if none left the collimators), whether it
    scattered in a slab, and how many source photons the history drew."""
    m = _Marshalled(problem, physics, field)
    X, Y, E = np.empty(n), np.empty(n), np.empty(n)
    coll = np.empty(n, dtype=np.int32)
    k = np.empty(n, dtype=np.int32)
    rc = lib().orc_sample_ps2_many(C.byref(m.s), int(seed), int(hist_begin), int(n), _dp(X), _dp(Y), _dp(E),
                                   coll.ctypes.data_as(C.POINTER(C.c_int32)), k.ctypes.data_as(C.POINTER(C.c_int32)))
    if rc:
        raise RuntimeError("field has no source rectangle")
    return X, Y, E, coll.astype(bool), k


def tmap(problem, ix=None, iy=None, field=None):
    """Radiological thickness (cm) for EPID pixels; all pixels when ix is None."""
    m = _Marshalled(problem, field=field)
    if ix is None:
        yy, xx = np.meshgrid(np.arange(m.s.npy), np.arange(m.s.npx), indexing="ij")
        ix, iy = xx.ravel(), yy.ravel()
        shape = (m.s.npy, m.s.npx)
    else:
        shape = np.shape(ix)
    ix = np.ascontiguousarray(ix, dtype=np.int32).ravel()
    iy = np.ascontiguousarray(iy, dtype=np.int32).ravel()
    t = np.empty(ix.size, dtype=np.float64)
    lib().orc_tmap(C.byref(m.s), ix.ctypes.data_as(C.POINTER(C.c_int32)),
                   iy.ctypes.data_as(C.POINTER(C.c_int32)), ix.size, _dp(t))
    return t.reshape(shape)


def siddon_ray(problem, p1, p2):
    m = _Marshalled(problem)
    a = np.ascontiguousarray(p1, dtype=np.float64)
    b = np.ascontiguousarray(p2, dtype=np.float64)
    return lib().orc_siddon_ray(C.byref(m.s), _dp(a), _dp(b))


def gamma(ref, ev, pixel_mm, dd=0.01, dta_mm=1.0, threshold=0.10, step_mm=None, radius_mm=None):
    """Global gamma pass rate of `ev` against `ref` (the form used in Sec. 2.3.3)."""
    ref = np.ascontiguousarray(ref, dtype=np.float64)
    ev = np.ascontiguousarray(ev, dtype=np.float64)
    ny, nx = ref.shape
    h = step_mm if step_mm is not None else min(pixel_mm, dta_mm / 10.0)
    rad = radius_mm if radius_mm is not None else 3.0 * dta_mm
    g = np.empty_like(ref)
    rate = lib().orc_gamma(_dp(ref), _dp(ev), nx, ny, float(pixel_mm), float(dd), float(dta_mm),
                           float(threshold), float(h), float(rad), _dp(g))
    return rate, g


# --------------------------------------------------------------------------
# Closed-form steps in numpy (FP64)
# --------------------------------------------------------------------------

def hu_to_rho_mat(hu):
    """HU -> (density, material) per the stated curve, through the C routine."""
    hu = np.asarray(hu).ravel()
    rho = np.empty(hu.size)
    mat = np.empty(hu.size, dtype=np.int32)
    r, mm = C.c_double(), C.c_int()
    for i, v in enumerate(hu):
        lib().orc_hu_to_rho_mat(int(v), C.byref(r), C.byref(mm))
        rho[i], mat[i] = r.value, mm.value
    return rho, mat


def aperture_bbox(field):
    """Bounding rectangle (a along X, b along Y) of the union of open apertures (Sec. 2.2)."""
    x0 = y0 = np.inf
    x1 = y1 = -np.inf
    for k in range(field.leaves.shape[0]):
        jx1, jx2, jy1, jy2 = field.jaws[k]
        for j in range(field.leaves.shape[1]):
            lx = max(field.leaves[k, j, 0], jx1)
            rx = min(field.leaves[k, j, 1], jx2)
            ly = max(field.pair_edges[j], jy1)
            ry = min(field.pair_edges[j + 1], jy2)
            if rx > lx and ry > ly and field.mu[k] > 0:
                x0, x1, y0, y1 = min(x0, lx), max(x1, rx), min(y0, ly), max(y1, ry)
    return x1 - x0, y1 - y0


def effective_field_size(field, literal=False):
    """Eq. 1.  As printed, s = ab / (2(a+b)) gives 2.5 cm for a 10x10 field, which
    cannot index Table 1; the reading used is the equivalent square 2ab/(a+b)."""
    a, b = aperture_bbox(field)
    return a * b / (2.0 * (a + b)) if literal else 2.0 * a * b / (a + b)


def lut_k(lut, t, s):
    """Bilinear k(t, s) on the node grids, clamped at the edges (Sec. 3.1)."""
    tn, sn, K = np.asarray(lut.t_nodes, float), np.asarray(lut.s_nodes, float), np.asarray(lut.k, float)
    t = np.clip(np.asarray(t, float), tn[0], tn[-1])
    s = float(np.clip(s, sn[0], sn[-1]))
    it = np.clip(np.searchsorted(tn, t, side="right") - 1, 0, tn.size - 2)
    js = int(np.clip(np.searchsorted(sn, s, side="right") - 1, 0, sn.size - 2))
    ft = (t - tn[it]) / (tn[it + 1] - tn[it])
    fs = (s - sn[js]) / (sn[js + 1] - sn[js])
    k00, k01 = K[js, it], K[js, it + 1]
    k10, k11 = K[js + 1, it], K[js + 1, it + 1]
    return (1 - fs) * ((1 - ft) * k00 + ft * k01) + fs * ((1 - ft) * k10 + ft * k11)


def patient_dose(vox_mev, phantom, n_hist):
    """Per-history dose (Gy) of each CT voxel from its deposited energy (MeV):
    E / (rho V), rho from the HU curve, V the voxel volume."""
    rho, _ = hu_to_rho_mat(phantom.hu)
    vol = phantom.vox[0] * phantom.vox[1] * phantom.vox[2]
    vox_mev = np.asarray(vox_mev, dtype=np.float64)
    return vox_mev * 1.602176634e-13 / (rho.reshape(vox_mev.shape) * vol * 1e-3) / float(n_hist)


def resample(src, src_pitch, dnx, dny, dst_pitch):
    """Bilinear resampling onto another pixel grid centred on the same axis:
    destination centre X = ((i + 1/2) - n/2) pitch is looked up at source
    index X / src_pitch + snx/2 - 1/2, clamped to the outer source centres."""
    src = np.asarray(src, dtype=np.float64)
    sny, snx = src.shape
    X = ((np.arange(dnx) + 0.5) - 0.5 * dnx) * dst_pitch
    Y = ((np.arange(dny) + 0.5) - 0.5 * dny) * dst_pitch
    fx = np.clip(X / src_pitch + 0.5 * snx - 0.5, 0, snx - 1)
    fy = np.clip(Y / src_pitch + 0.5 * sny - 0.5, 0, sny - 1)
    x0 = np.floor(fx).astype(int)
    y0 = np.floor(fy).astype(int)
    x1 = np.minimum(x0 + 1, snx - 1)
    y1 = np.minimum(y0 + 1, sny - 1)
    ax = (fx - x0)[None, :]
    ay = (fy - y0)[:, None]
    return ((1 - ay) * ((1 - ax) * src[y0][:, x0] + ax * src[y0][:, x1]) +
            ay * ((1 - ax) * src[y1][:, x0] + ax * src[y1][:, x1]))


def plan_image(doses, tmaps, fields, lut, weights=None):
    """Weighted sums over control points / fields: sum_f w_f D_f and
    sum_f w_f k(t_f, s_f) D_f (Sec. 3.1 per field)."""
    F = len(doses)
    w = np.full(F, 1.0 / F) if weights is None else np.asarray(weights, dtype=np.float64)
    dose = sum(w[f] * np.asarray(doses[f]) for f in range(F))
    sig = sum(w[f] * lut_k(lut, tmaps[f], effective_field_size(fields[f])) * np.asarray(doses[f]) for f in range(F))
    return dose, sig


def batch_counts(n_hist, B, hist_begin=0):
    """Number of history ids h in [hist_begin, hist_begin+n) with h mod B == b."""
    ids = np.arange(B)
    first = (ids - hist_begin) % B
    return np.where(first < n_hist, (n_hist - first + B - 1) // B, 0).astype(np.int64)


def dose_stats(tally_mev, n_hist, epid, hist_begin=0):
    """Per-history dose (Gy) in the sensitive layer, its batch standard error and
    the mean relative uncertainty over pixels above half the maximum."""
    tally_mev = np.asarray(tally_mev, dtype=np.float64)
    B = tally_mev.shape[0]
    _, thick, rho = epid.layers[epid.sensitive]
    mass_kg = rho * epid.pitch * epid.pitch * thick * 1e-3
    conv = 1.602176634e-13 / mass_kg
    nb = batch_counts(n_hist, B, hist_begin).astype(np.float64)
    mean = tally_mev.sum(axis=0) / n_hist * conv
    with np.errstate(invalid="ignore", divide="ignore"):
        dbat = tally_mev / nb[:, None, None] * conv
    sigma = np.sqrt(((dbat - mean[None]) ** 2).sum(axis=0) / (B * (B - 1)))
    sel = mean > 0.5 * mean.max() if mean.max() > 0 else np.zeros_like(mean, dtype=bool)
    u = float(np.mean(sigma[sel] / mean[sel])) if sel.any() else float("nan")
    return mean, sigma, u
