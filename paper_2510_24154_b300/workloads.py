"""Seeded synthetic inputs for the EPID transit Monte Carlo path.

This module builds inputs only: HU phantoms, MLC-shaped IMRT fields, the EPID
layer stack, correction lookup tables and the transport settings.  It holds
none of the transport, ray-tracing or correction arithmetic, so both the CUDA
path and the FP64 oracle can take their inputs from it without sharing any of
the method's code.

Coordinates are in cm and energies in MeV.  The patient frame follows the CT
array: x (left-right) is the fastest index, y (anterior-posterior) the middle
one and z (cranio-caudal) the slowest, so an HU volume has shape [nz][ny][nx].
At gantry angle 0 the beam travels along +y; the gantry turns about z.

The paper's clinical inputs (CT, RTPLAN, measured images; Sec. 2.3) are not
available, so these generators stand in for them with the geometries the
paper states: SSD 90 cm over a 20 cm water slab (Sec. 2.3.1), SAD 100 cm and
SID 150 cm (Sec. 2.3.2), a 60-pair MLC and EPID pixel grids (Sec. 2.3.3).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# Material ids shared by the C-ABI and the oracle's input structs.
MAT_AIR, MAT_LUNG, MAT_WATER, MAT_BONE, MAT_CU, MAT_GOS, MAT_SI = range(7)
MATERIAL_NAMES = ("air", "lung", "water", "bone", "copper", "Gd2O2S", "a-Si")


@dataclass
class Phantom:
    """CT volume: int16 HU [nz][ny][nx], voxel size and the box's lower corner."""
    hu: np.ndarray
    vox: tuple
    origin: tuple

    @property
    def shape_xyz(self):
        nz, ny, nx = self.hu.shape
        return nx, ny, nz


@dataclass
class Epid:
    """Multi-layer EPID slab (Sec. 2.1.3), layers listed from the source side.

    Each layer is (material id, thickness cm, density g/cm^3).  The sensitive
    layer's centre lies on the plane at SID from the source; pixels tile the
    layer laterally, npx along the beam-frame X axis and npy along Y.
    """
    layers: list
    sensitive: int
    npx: int
    npy: int
    pitch: float


@dataclass
class Field:
    """One static IMRT field: MLC segments at the isocentre plane.

    pair_edges: [n_pairs+1] leaf-pair boundaries along beam-frame Y.
    leaves:     [n_seg][n_pairs][2] (left, right) leaf tips along X.
    jaws:       [n_seg][4] (x1, x2, y1, y2).
    mu:         [n_seg] monitor-unit weights.
    leaf_transmission: fraction of the open fluence that passes closed
                leaves (0 = ideal MLC).
    jaw_transmission: fraction that passes the jaws (0 = opaque).
    tg_width:   tongue-and-groove strip width at the isocentre plane (cm):
                within half of it from a pair boundary, the opening is the
                intersection of both pairs' openings.
    leaf_gap:   dosimetric leaf gap (cm): an open pair's effective opening
                is wider by this much (rounded leaf ends).
    leaf_thickness, jaw_thickness: tungsten slab thickness along the beam
                (cm) of the leaves (top 51 cm from the source) and of the
                jaws (top 28 cm); either > 0 transports the source photons
                through the collimators (phase space 2 of Sec. 2.1.1) in
                place of the transmission factors, which must then be 0.
    """
    pair_edges: np.ndarray
    leaves: np.ndarray
    jaws: np.ndarray
    mu: np.ndarray
    gantry_deg: float = 0.0
    sad: float = 100.0
    sid: float = 150.0
    iso: tuple = (0.0, 0.0, 0.0)
    leaf_transmission: float = 0.0
    jaw_transmission: float = 0.0
    tg_width: float = 0.0
    leaf_gap: float = 0.0
    leaf_thickness: float = 0.0
    jaw_thickness: float = 0.0


@dataclass
class Lut:
    """k(t, s) table: k[is][it] over strictly increasing node axes (Sec. 3.1)."""
    t_nodes: np.ndarray
    s_nodes: np.ndarray
    k: np.ndarray
    k_scale: float = 1.0
    t_offset: float = 0.0
    eq1_literal: bool = False


@dataclass
class Physics:
    """Transport settings (Sec. 2.1.2 cutoffs; the rest are stated readings)."""
    coupled: bool = True
    e_max: float = 6.0          # spectrum end point, MeV
    mono_energy: float = 0.0    # > 0: monoenergetic source instead of the spectrum
    photon_cutoff: float = 0.01
    electron_cutoff: float = 0.2
    wcc: float = 0.2
    wcb: float = 0.01
    step_fraction: float = 0.05
    n_batches: int = 16
    max_steps: int = 10000


@dataclass
class Problem:
    """Everything one simulation needs."""
    name: str
    phantom: Phantom
    epid: Epid
    field: Field
    lut: Lut
    physics: Physics
    n_histories: int
    seed: int
    extra: dict = field(default_factory=dict)


# ---------------------------------------------------------------------------
# MLC, fields, EPID
# ---------------------------------------------------------------------------

def millennium_pair_edges() -> np.ndarray:
    """60 leaf pairs at the isocentre: 10 x 1 cm, 40 x 0.5 cm, 10 x 1 cm."""
    edges = [-20.0 + i for i in range(11)]                    # -20 .. -10
    edges += [-10.0 + 0.5 * i for i in range(1, 41)]          # -9.5 .. 10
    edges += [10.0 + i for i in range(1, 11)]                 # 11 .. 20
    e = np.array(edges, dtype=np.float64)
    assert e.size == 61
    return e


def open_field(size_x: float, size_y: float, gantry_deg: float = 0.0,
               sad: float = 100.0, sid: float = 150.0, iso=(0.0, 0.0, 0.0)) -> Field:
    """A single rectangular segment, leaves at +-size_x/2 and Y jaws at +-size_y/2."""
    edges = millennium_pair_edges()
    n_pairs = edges.size - 1
    leaves = np.zeros((1, n_pairs, 2))
    leaves[0, :, 0] = -size_x / 2
    leaves[0, :, 1] = size_x / 2
    jaws = np.array([[-size_x / 2, size_x / 2, -size_y / 2, size_y / 2]])
    return Field(edges, leaves, jaws, np.array([1.0]), gantry_deg, sad, sid, tuple(iso))


def imrt_field(rng: np.random.Generator, n_seg: int, gantry_deg: float = 0.0,
               sad: float = 100.0, sid: float = 150.0, iso=(0.0, 0.0, 0.0),
               leaf_range: float = 10.0, jaw_y: float = 10.0) -> Field:
    """Random MLC segments: each pair's two tips U(-r, r) sorted; MU ~ Dirichlet(1)."""
    edges = millennium_pair_edges()
    n_pairs = edges.size - 1
    tips = rng.uniform(-leaf_range, leaf_range, size=(n_seg, n_pairs, 2))
    tips.sort(axis=2)
    mu = rng.exponential(1.0, size=n_seg)
    mu /= mu.sum()
    jaws = np.tile(np.array([-leaf_range, leaf_range, -jaw_y, jaw_y]), (n_seg, 1))
    return Field(edges, tips, jaws, mu, gantry_deg, sad, sid, tuple(iso))


def epid_default(npx: int, npy: int, pitch: float, gos_density: float = 7.34) -> Epid:
    """1 mm Cu build-up, 0.29 mm Gd2O2S (sensitive), 1 mm a-Si."""
    layers = [(MAT_CU, 0.1, 8.96), (MAT_GOS, 0.029, gos_density), (MAT_SI, 0.1, 2.33)]
    return Epid(layers, 1, npx, npy, pitch)


# ---------------------------------------------------------------------------
# Phantoms
# ---------------------------------------------------------------------------

def water_slab(nx=64, ny=40, nz=64, vox=0.5) -> Phantom:
    """Homogeneous water (0 HU) box centred on the isocentre.

    The 40-voxel (20 cm) axis is y, the beam axis at gantry 0, so the entrance
    surface sits at SSD 90 cm as in Sec. 2.3.1.
    """
    hu = np.zeros((nz, ny, nx), dtype=np.int16)
    origin = (-nx * vox / 2, -ny * vox / 2, -nz * vox / 2)
    return Phantom(hu, (vox, vox, vox), origin)


def _centres(n, vox, lo):
    return lo + (np.arange(n) + 0.5) * vox


def thorax_ct(rng: np.random.Generator, nx=256, ny=256, nz=128, vox=0.2,
              jitter: float = 0.0, noise_hu: float = 20.0) -> Phantom:
    """Synthetic thorax-like CT centred on the isocentre.

    Water ellipse (0 HU) with semi-axes 15 cm (x) by 10 cm (y) extruded along
    z, air (-1000 HU) outside; three bone rods (+1000 HU, radius 1 cm) along z;
    two lung ellipsoids (-750 HU, semi-axes 4 x 3 x 8 cm); i.i.d. Gaussian
    noise; values clamped to [-1024, 3071].  `jitter` scales random +-fraction
    perturbations of sizes and positions (the denoiser's training phantoms).
    """
    def j(v):
        return v * (1.0 + jitter * rng.uniform(-1, 1)) if jitter else v

    ox, oy, oz = -nx * vox / 2, -ny * vox / 2, -nz * vox / 2
    x = _centres(nx, vox, ox)[None, None, :]
    y = _centres(ny, vox, oy)[None, :, None]
    z = _centres(nz, vox, oz)[:, None, None]
    ax, ay = j(15.0), j(10.0)
    hu = np.full((nz, ny, nx), -1000.0)
    body = (x / ax) ** 2 + (y / ay) ** 2 <= 1.0
    hu = np.where(body, 0.0, hu)
    for (cx, cy) in ((0.0, 6.5), (-9.0, 0.0), (9.0, 0.0)):
        cx, cy, r = j(cx), j(cy), j(1.0)
        rod = (x - cx) ** 2 + (y - cy) ** 2 <= r * r
        hu = np.where(rod & body, 1000.0, hu)
    for sx in (-1.0, 1.0):
        cx, cy, cz = sx * j(6.0), j(-1.0), 0.0
        a, b, c = j(4.0), j(3.0), j(8.0)
        lung = ((x - cx) / a) ** 2 + ((y - cy) / b) ** 2 + ((z - cz) / c) ** 2 <= 1.0
        hu = np.where(lung & body, -750.0, hu)
    hu = hu + rng.normal(0.0, noise_hu, size=hu.shape)
    hu = np.clip(np.rint(hu), -1024, 3071).astype(np.int16)
    return Phantom(hu, (vox, vox, vox), (ox, oy, oz))


def anthropomorphic_ct(rng: np.random.Generator, nx=512, ny=512, nz=200, vox=0.1,
                       noise_hu: float = 20.0, jitter: float = 0.0) -> Phantom:
    """Larger thorax-like phantom: body outline, spine, rib arcs, lungs, organs.
    `jitter` scales random +-fraction perturbations of sizes and positions (the
    denoiser's training phantoms); at 0 no random number is drawn for them."""
    def j(v):
        return v * (1.0 + jitter * rng.uniform(-1, 1)) if jitter else v

    ox, oy, oz = -nx * vox / 2, -ny * vox / 2, -nz * vox / 2
    x = _centres(nx, vox, ox)[None, None, :]
    y = _centres(ny, vox, oy)[None, :, None]
    z = _centres(nz, vox, oz)[:, None, None]
    hu = np.full((nz, ny, nx), -1000.0, dtype=np.float32)
    bx, by = j(17.0), j(11.0)
    body = (x / bx) ** 2 + (y / by) ** 2 <= 1.0
    hu = np.where(body, 0.0, hu)
    for sx in (-1.0, 1.0):
        cx, cy, a, b, c = sx * j(7.0), j(-0.5), j(5.0), j(6.5), j(9.0)
        lung = ((x - cx) / a) ** 2 + ((y - cy) / b) ** 2 + (z / c) ** 2 <= 1.0
        hu = np.where(lung & body, -750.0, hu)
    cx, cy, cz, a, b, c = j(1.0), j(-3.0), j(2.0), j(4.0), j(3.5), j(5.0)
    organs = (((x - cx) / a) ** 2 + ((y - cy) / b) ** 2 + ((z - cz) / c) ** 2 <= 1.0)
    hu = np.where(organs & body, 40.0, hu)
    sy, sr = j(7.5), j(1.6)
    spine = (x ** 2 + (y - sy) ** 2 <= sr ** 2)
    hu = np.where(spine & body, 1000.0, hu)
    rr = (x / (bx - 1.2)) ** 2 + (y / (by - 1.2)) ** 2
    shell = (rr >= 0.86) & (rr <= 0.95)
    ribs = shell & (np.cos(2 * np.pi * z / j(2.5)) > 0.3) & body
    hu = np.where(ribs, 700.0, hu)
    hu = hu + rng.normal(0.0, noise_hu, size=hu.shape).astype(np.float32)
    hu = np.clip(np.rint(hu), -1024, 3071).astype(np.int16)
    return Phantom(hu, (vox, vox, vox), (ox, oy, oz))


# ---------------------------------------------------------------------------
# Correction tables
# ---------------------------------------------------------------------------

TABLE1_T = np.array([0.0, 5.0, 10.0, 15.0, 20.0])
TABLE1_S = np.array([5.0, 10.0, 15.0, 20.0])
# Table 1 of the paper (Sec. 3.1): rows are square field sizes, columns thicknesses.
TABLE1_K = np.array([
    [0.999, 0.974, 0.960, 0.949, 0.949],
    [1.001, 0.975, 0.967, 0.964, 0.953],
    [0.995, 0.982, 0.983, 0.996, 0.986],
    [0.991, 0.997, 1.015, 1.034, 1.043],
])


def lut_table1() -> Lut:
    return Lut(TABLE1_T.copy(), TABLE1_S.copy(), TABLE1_K.copy())


def lut_bilinear(nt=64, ns=32) -> Lut:
    """k = 1 + 0.1 ((s-16)/14)(t/40): bilinear, so interpolation reproduces it exactly."""
    t = np.linspace(0.0, 40.0, nt)
    s = np.linspace(2.0, 30.0, ns)
    k = 1.0 + 0.1 * ((s[:, None] - 16.0) / 14.0) * (t[None, :] / 40.0)
    return Lut(t, s, k)


def lut_wavy(nt=64, ns=32) -> Lut:
    """The bilinear table plus a smooth non-bilinear ripple, clipped to [0.9, 1.1]."""
    base = lut_bilinear(nt, ns)
    ripple = 0.02 * np.sin(2 * np.pi * base.t_nodes[None, :] / 40.0) * \
        np.cos(2 * np.pi * (base.s_nodes[:, None] - 2.0) / 28.0)
    return Lut(base.t_nodes, base.s_nodes, np.clip(base.k + ripple, 0.9, 1.1))


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def config_water_open(n_histories=1_000_000, seed=0, npx=128, npy=128, pitch=0.3,
                      coupled=False, field_cm=10.0) -> Problem:
    """Photon-only, 6 MV spectrum, open 10x10 field, 64x40x64 water box at 5 mm,
    EPID 128x128 at 3 mm (the small single-field workload)."""
    return Problem(
        name="water_open_10x10",
        phantom=water_slab(),
        epid=epid_default(npx, npy, pitch),
        field=open_field(field_cm, field_cm),
        lut=lut_table1(),
        physics=Physics(coupled=coupled),
        n_histories=n_histories, seed=seed)


def config_paper_grid(n_histories=1_000_000_000, seed=0) -> Problem:
    """The small single-field workload coupled, scored on the EPID grid of the
    paper's image comparisons: 160 x 160 pixels at 2.5 mm (64 x 40 x 64 water
    at 5 mm, SSD 90, open 10 x 10 field)."""
    p = config_water_open(n_histories=n_histories, seed=seed, npx=160, npy=160, pitch=0.25, coupled=True)
    p.name = "water_open_10x10_paper_grid"
    return p


def config_thorax_imrt(n_histories=100_000_000, seed=1, scale=1, epid_scale=1,
                       n_seg=9, gantry_deg=0.0) -> Problem:
    """Coupled transport through the 256x256x128 thorax CT at 2 mm, one 9-segment
    IMRT field, EPID 1024x768 at 0.39 mm, 64x32 correction table.

    `scale` > 1 coarsens the CT by that factor (same physical box) and
    `epid_scale` > 1 coarsens the pixel grid, for oracle-sized parity cases.
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = 256 // scale, 256 // scale, 128 // scale
    ph = thorax_ct(rng, nx, ny, nz, 0.2 * scale)
    fld = imrt_field(rng, n_seg, gantry_deg)
    ep = epid_default(1024 // epid_scale, 768 // epid_scale, 0.039 * epid_scale)
    return Problem(
        name="thorax_imrt_9seg",
        phantom=ph, epid=ep, field=fld, lut=lut_bilinear(),
        physics=Physics(coupled=True),
        n_histories=n_histories, seed=seed)


def config_batched_plan(seed=2, n_fields=25, scale=1, epid_scale=1,
                        hist_lo=1e7, hist_hi=2e8):
    """25 fields of 5-40 segments each, gantry U[0,360), histories log-uniform."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = 256 // scale, 256 // scale, 128 // scale
    ph = thorax_ct(np.random.default_rng(1), nx, ny, nz, 0.2 * scale)
    ep = epid_default(1024 // epid_scale, 768 // epid_scale, 0.039 * epid_scale)
    fields, hist = [], []
    for _ in range(n_fields):
        n_seg = int(rng.integers(5, 41))
        g = float(rng.uniform(0.0, 360.0))
        fields.append(imrt_field(rng, n_seg, g))
        hist.append(int(math.exp(rng.uniform(math.log(hist_lo), math.log(hist_hi)))))
    return ph, ep, fields, hist


def vmat_arc(rng: np.random.Generator, n_cp: int = 64, start_deg: float = 181.0, arc_deg: float = 358.0,
             leaf_range: float = 8.0, jaw_y: float = 8.0, step_cm: float = 0.5):
    """A VMAT arc: n_cp control points, gantry from start_deg over arc_deg
    (clockwise), one aperture each whose leaf tips follow a bounded random
    walk (steps N(0, step_cm)) so that neighbouring apertures are alike;
    MU per control point ~ 0.5 + U(0, 1), normalised.  Returns the control
    points as single-segment fields and their MU fractions."""
    edges = millennium_pair_edges()
    n_pairs = edges.size - 1
    tips = np.sort(rng.uniform(-leaf_range / 2, leaf_range / 2, size=(n_pairs, 2)), axis=1)
    mu = 0.5 + rng.uniform(0.0, 1.0, size=n_cp)
    mu /= mu.sum()
    fields = []
    for k in range(n_cp):
        tips = np.clip(tips + rng.normal(0.0, step_cm, size=tips.shape), -leaf_range, leaf_range)
        tips.sort(axis=1)
        tips[:, 1] = np.maximum(tips[:, 1], tips[:, 0] + 0.2)       # keep every pair open
        g = (start_deg + arc_deg * k / max(n_cp - 1, 1)) % 360.0
        jaws = np.array([[-leaf_range, leaf_range, -jaw_y, jaw_y]])
        fields.append(Field(edges, tips[None].copy(), jaws, np.ones(1), g))
    return fields, mu


def config_vmat(n_cp: int = 64, seed: int = 5, scale: int = 1, epid_npx: int = 1190, epid_pitch: float = 0.0336):
    """VMAT arc on the thorax CT, imaged by the 1190 x 1190 EPID at 0.336 mm
    (the paper's detector, Sec. 2.3)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = 256 // scale, 256 // scale, 128 // scale
    ph = thorax_ct(np.random.default_rng(1), nx, ny, nz, 0.2 * scale)
    fields, mu = vmat_arc(rng, n_cp)
    return ph, epid_default(epid_npx, epid_npx, epid_pitch), fields, mu


def config_anthropomorphic(n_histories=1_000_000_000, seed=4) -> Problem:
    """512x512x200 at 1 mm, one 40-segment field, EPID 1190x1190 at 0.336 mm."""
    rng = np.random.default_rng(seed)
    ph = anthropomorphic_ct(rng)
    fld = imrt_field(rng, 40)
    return Problem(
        name="anthropomorphic_40seg",
        phantom=ph, epid=epid_default(1190, 1190, 0.0336), field=fld,
        lut=lut_bilinear(), physics=Physics(coupled=True),
        n_histories=n_histories, seed=seed)


# ------------------------------------------------------------ denoiser ----

def unet_params(layer_shapes, seed=0, bias_sd=0.05):
    """Seeded parameter vector for a network given as (name, Co, k, Ci)
    tuples: per layer He-normal weights [Co][k][k][Ci] (sd sqrt(2 / (k k Ci)))
    then biases N(0, bias_sd), float32."""
    rng = np.random.default_rng(seed)
    parts = []
    for _, co, k, ci in layer_shapes:
        parts.append(rng.normal(size=co * k * k * ci) * np.sqrt(2.0 / (k * k * ci)))
        parts.append(rng.normal(size=co) * bias_sd)
    return np.concatenate(parts).astype(np.float32)


def bf16_values(rng, shape, scale=1.0, nonneg=False):
    """Random float32 values that are exactly representable in bfloat16."""
    a = rng.normal(size=shape) * scale
    if nonneg:
        a = np.abs(a)
    u = a.astype(np.float32).view(np.uint32) & np.uint32(0xFFFF0000)
    return u.view(np.float32)
