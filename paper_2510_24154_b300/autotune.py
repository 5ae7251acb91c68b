"""Launch-shape autotuner for the transport kernels.

Picks, per device and workload, the launch settings of a run -- the
occupancy build of each transport kernel (2, 3 or 4 CTAs of 256 threads per
SM), the block size, the particle-bank capacity, the number of new histories
admitted per wave and the graph-driven wave loop -- that give the most
histories per second on a short timed run.  None of these settings changes a
result: a history's random numbers are keyed by its id and the tallies are
integer sums, so every candidate produces the same tally bit for bit and only
the time differs.

The search is a coordinate descent from the library defaults: each knob in
turn is set to each of its candidate values with the others fixed, and the
fastest value is kept.  Results are cached in a JSON file keyed by the GPU
(name and SM count) and the workload's shape; a cached entry is returned
without timing anything.
"""
from __future__ import annotations

import hashlib
import json
import os
from pathlib import Path
from typing import Callable, Dict, Iterable, Optional

DEFAULTS = {"regs_variant": (4, 4, 4, 4), "block_size": 256, "bank_capacity": 1 << 23, "primaries_per_wave": 0,
            "use_graph": 0}

SEARCH = {
    "regs_variant": [(4, 4, 4, 4), (4, 3, 4, 3), (4, 3, 4, 4), (3, 3, 4, 4), (3, 3, 3, 3), (4, 2, 4, 4)],
    "block_size": [256, 128],
    "bank_capacity": [1 << 23, 1 << 24],
    "primaries_per_wave": [0, 1 << 20, 1 << 22],
    "use_graph": [0, 1],
}


def cache_path() -> Path:
    env = os.environ.get("ARCHER_EPID_AUTOTUNE_CACHE")
    if env:
        return Path(env)
    return Path(os.environ.get("XDG_CACHE_HOME", Path.home() / ".cache")) / "archer_epid" / "autotune.json"


def workload_key(device_name: str, sm_count: int, problem, n_fields: int = 1) -> str:
    """The GPU and the shape of the work: CT and EPID grids, physics mode and
    the number of fields (the history count does not enter: rates are per
    history)."""
    ph, ep, phys = problem.phantom, problem.epid, problem.physics
    sig = {
        "gpu": device_name, "sms": int(sm_count), "ct": list(ph.hu.shape), "vox": [round(v, 6) for v in ph.vox],
        "epid": [ep.npx, ep.npy, round(ep.pitch, 6), len(ep.layers)], "coupled": bool(phys.coupled),
        "mono": float(phys.mono_energy), "cut": [phys.photon_cutoff, phys.electron_cutoff],
        "batches": phys.n_batches, "fields": int(n_fields),
    }
    return hashlib.sha1(json.dumps(sig, sort_keys=True).encode()).hexdigest()[:16]


def _load(path: Path) -> dict:
    try:
        return json.loads(path.read_text())
    except (OSError, ValueError):
        return {}


def _store(path: Path, key: str, entry: dict) -> None:
    path.parent.mkdir(parents=True, exist_ok=True)
    data = _load(path)
    data[key] = entry
    tmp = path.with_suffix(".tmp")
    tmp.write_text(json.dumps(data, indent=1, sort_keys=True))
    tmp.replace(path)


def coordinate_descent(timer: Callable[[dict], float], search: Optional[Dict[str, Iterable]] = None,
                       start: Optional[dict] = None, sweeps: int = 1):
    """Minimises timer(settings) (seconds per history) one knob at a time.
    Returns (best settings, best time, {repr(settings): time} of every trial)."""
    search = SEARCH if search is None else search
    best = dict(DEFAULTS if start is None else start)
    trials: Dict[str, float] = {}

    def measure(cfg):
        k = json.dumps({a: list(b) if isinstance(b, tuple) else b for a, b in sorted(cfg.items())})
        if k not in trials:
            trials[k] = float(timer(dict(cfg)))
        return trials[k]

    best_t = measure(best)
    for _ in range(sweeps):
        changed = False
        for knob, values in search.items():
            for v in values:
                cand = dict(best)
                cand[knob] = v
                t = measure(cand)
                if t < best_t:
                    best, best_t, changed = cand, t, True
        if not changed:
            break
    return best, best_t, trials


def gpu_timer(problem, fields=None, n_histories: int = 2_000_000, device: int = 0, seed: int = 1):
    """A timer for coordinate_descent: seconds per history of one run of
    `n_histories` (per field) on `problem` (or its batch `fields`), after one
    short warm-up run, with the given launch settings."""
    from .binding import Simulator

    def timer(settings: dict) -> float:
        kw = dict(settings)
        kw["regs_variant"] = list(kw["regs_variant"])
        sim = Simulator(problem.physics, device=device, **kw)
        try:
            sim.init_geometry(problem.phantom, problem.epid)
            if fields is None:
                sim.set_field(problem.field, problem.lut)
                sim.run(max(n_histories // 20, 1000), seed)
                st = sim.run(n_histories, seed)
                return st["gpu_ms"] * 1e-3 / n_histories
            sim.set_fields(fields, problem.lut)
            sim.run_batch([max(n_histories // 20, 1000)] * len(fields), seed)
            st = sim.run_batch([n_histories] * len(fields), seed)
            return st["gpu_ms"] * 1e-3 / (n_histories * len(fields))
        finally:
            sim.close()

    return timer


def autotune(problem, fields=None, n_histories: int = 2_000_000, device: int = 0, search=None,
             path: Optional[Path] = None, retune: bool = False, timer=None) -> dict:
    """Best launch settings for `problem` on GPU `device` (cached).  Returns a
    dict of Simulator keyword overrides plus the measured rate."""
    path = cache_path() if path is None else Path(path)
    if timer is None:
        import torch
        props = torch.cuda.get_device_properties(device)
        name, sms = props.name, props.multi_processor_count
        timer = gpu_timer(problem, fields, n_histories, device)
    else:
        name, sms = "custom-timer", 0
    key = workload_key(name, sms, problem, 1 if fields is None else len(fields))
    if not retune:
        hit = _load(path).get(key)
        if hit is not None:
            return hit
    best, best_t, trials = coordinate_descent(timer, search)
    entry = {k: (list(v) if isinstance(v, tuple) else v) for k, v in best.items()}
    entry["histories_per_s"] = 1.0 / best_t if best_t > 0 else None
    entry["trials"] = len(trials)
    _store(path, key, entry)
    return entry


def overrides(entry: dict) -> dict:
    """The Simulator keyword arguments of a cached entry."""
    return {k: entry[k] for k in DEFAULTS if k in entry}
