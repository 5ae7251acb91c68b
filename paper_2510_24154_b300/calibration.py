"""The simulated half of the dose-response calibration (Sec. 2.2, Eq. 2,
Table 1): S(t, s), the mean per-history EPID dose in the central 1 cm x 1 cm
of the image behind a water slab of thickness t for a square open field of
side s, computed with the transport library; k(t, s) = M(t, s) / S(t, s) once
the measured signals M are supplied (the measurements themselves are not
reproducible here).

Stated readings: the slab is water (0 HU), 40 cm x 40 cm laterally, centred
on the isocentre with the beam along its thickness (gantry 0); t = 0 is an
empty (air) geometry -- the paper's t = 0 includes the treatment couch, which
is not modelled; the field is an open s x s square at the isocentre; the
region is the pixels whose centres lie within 0.5 cm of the image centre.
S is expressed per unit primary fluence at the isocentre plane (the
per-history dose times the field area s^2, in Gy cm^2), as a fixed number of
monitor units delivers a fixed fluence whatever the field size; each point
runs histories_per_cm2 x s^2 histories, so all points carry similar
statistics.  The uncertainty of each S is the batch standard error of the
region mean.  Both come from the library (mc_get_region_dose) on the device.
"""
from __future__ import annotations

import numpy as np

from . import workloads as W

T_NODES = (0.0, 5.0, 10.0, 15.0, 20.0)
S_NODES = (5.0, 10.0, 15.0, 20.0)


def slab_phantom(t_cm: float, lateral_cm: float = 40.0, vox: float = 0.5) -> W.Phantom:
    """Water slab of thickness t along y (the beam at gantry 0), centred on
    the isocentre; t = 0 gives one voxel of air."""
    nxz = int(round(lateral_cm / vox))
    ny = max(int(round(t_cm / vox)), 1)
    hu = np.zeros((nxz, ny, nxz), dtype=np.int16) if t_cm > 0 else np.full((nxz, 1, nxz), -1000, dtype=np.int16)
    origin = (-nxz * vox / 2, -ny * vox / 2, -nxz * vox / 2)
    return W.Phantom(hu, (vox, vox, vox), origin)


def central_rect(epid: W.Epid, half_cm: float = 0.5):
    """Pixel rectangle [ix0, ix1) x [iy0, iy1) of the pixels whose centres lie
    within half_cm of the image centre in x and in y."""
    def span(n):
        c = ((np.arange(n) + 0.5) - n / 2) * epid.pitch
        idx = np.nonzero(np.abs(c) <= half_cm)[0]
        if idx.size == 0:
            raise ValueError("no pixel centre within the region")
        return int(idx[0]), int(idx[-1]) + 1
    (ix0, ix1), (iy0, iy1) = span(epid.npx), span(epid.npy)
    return ix0, ix1, iy0, iy1


def central_region(epid: W.Epid, half_cm: float = 0.5):
    """The same region as a boolean mask [npy][npx]."""
    ix0, ix1, iy0, iy1 = central_rect(epid, half_cm)
    m = np.zeros((epid.npy, epid.npx), dtype=bool)
    m[iy0:iy1, ix0:ix1] = True
    return m


def s_table(histories_per_cm2: float = 1e6, t_nodes=T_NODES, s_nodes=S_NODES, epid: W.Epid | None = None,
            seed: int = 11, device: int = 0, physics: W.Physics | None = None):
    """S(t, s) and its uncertainty, arrays [len(s_nodes)][len(t_nodes)] in
    Gy cm^2 per history (the layout of Table 1: rows field sizes, columns
    thicknesses)."""
    from .binding import Simulator
    epid = epid or W.epid_default(1024, 768, 0.039)
    physics = physics or W.Physics(coupled=True)
    rect = central_rect(epid)
    S = np.zeros((len(s_nodes), len(t_nodes)))
    U = np.zeros_like(S)
    sim = Simulator(physics, device=device)
    try:
        for j, t in enumerate(t_nodes):
            sim.init_geometry(slab_phantom(t), epid)
            for i, s in enumerate(s_nodes):
                n = int(round(histories_per_cm2 * s * s))
                sim.set_field(W.open_field(s, s))
                done = 0
                while done < n:
                    k = min(n - done, 1 << 31)
                    sim.run(k, seed + 1000 * j + i)
                    done += k
                m, u = sim.region_dose(*rect)
                S[i, j], U[i, j] = m * s * s, u * s * s
    finally:
        sim.close()
    return S, U


def k_table(measured: np.ndarray, simulated: np.ndarray, t_nodes=T_NODES, s_nodes=S_NODES,
            k_scale: float = 1.0) -> W.Lut:
    """Eq. 2: k(t, s) = M(t, s) / S(t, s) on the calibration nodes, as the
    table the correction step interpolates (rows s, columns t)."""
    M = np.asarray(measured, dtype=np.float64)
    S = np.asarray(simulated, dtype=np.float64)
    if M.shape != S.shape or M.shape != (len(s_nodes), len(t_nodes)):
        raise ValueError("M and S must be [len(s_nodes)][len(t_nodes)]")
    return W.Lut(np.asarray(t_nodes, float), np.asarray(s_nodes, float), M / S, k_scale=k_scale)
