"""Shared helpers for the GPU parity tests: build both sides from one seeded
Problem and compare their images.  Holds no transport arithmetic."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2510_24154_b300 import workloads as W

QUANTA_PER_MEV = 2.56e8


def water_case(n=1_000_000, coupled=False, npx=64, pitch=0.6, batches=16, field_cm=10.0):
    p = W.config_water_open(n_histories=n, npx=npx, npy=npx, pitch=pitch, coupled=coupled, field_cm=field_cm)
    p.physics.n_batches = batches
    return p


def thorax_case(n=300_000, scale=4, epid_scale=8, batches=16, gantry=0.0, seed=1):
    p = W.config_thorax_imrt(n_histories=n, scale=scale, epid_scale=epid_scale, gantry_deg=gantry, seed=seed)
    p.physics.n_batches = batches
    return p


def make_sim(problem, **overrides):
    from paper_2510_24154_b300.binding import Simulator
    sim = Simulator(problem.physics, **overrides)
    sim.init_geometry(problem.phantom, problem.epid)
    sim.set_field(problem.field, problem.lut)
    return sim


def gpu_run(problem, seed=None, n=None, **overrides):
    sim = make_sim(problem, **overrides)
    st = sim.run(problem.n_histories if n is None else n, problem.seed if seed is None else seed)
    tally = sim.tally().astype(np.float64) / QUANTA_PER_MEV
    return sim, st, tally


def sensitive_energy(res_tally):
    return float(res_tally.sum())


def three_sigma_fraction(d1, s1, d2, s2, threshold=0.10):
    """Fraction of pixels above `threshold` x max (of d2) with |d1-d2| <= 3 sqrt(s1^2+s2^2)."""
    sel = d2 > threshold * d2.max()
    ok = np.abs(d1 - d2)[sel] <= 3.0 * np.sqrt(s1 ** 2 + s2 ** 2)[sel]
    return float(ok.mean()), int(sel.sum())


def gamma_rate(ref, ev, pitch_cm, dd=0.01, dta_mm=1.0):
    rate, _ = oracle.gamma(ref, ev, pixel_mm=pitch_cm * 10.0, dd=dd, dta_mm=dta_mm, threshold=0.10)
    return rate


def energy_closure(st):
    out = st["e_ct"] + st["e_epid"].sum() + st["e_esc"] + st["e_lost"]
    return abs(out - st["e_src"]) / st["e_src"]
