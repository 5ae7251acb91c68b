"""Host logic of the launch-shape autotuner: the coordinate descent finds the
optimum of a separable cost, and the cache returns an entry without timing."""
import json

from paper_2510_24154_b300 import autotune as A
from paper_2510_24154_b300 import workloads as W


def _cost(cfg):
    # separable: best is regs (3,3,4,4), block 128, bank 2^24, ppw 2^20, graph on
    t = 1.0
    t += 0.0 if tuple(cfg["regs_variant"]) == (3, 3, 4, 4) else 0.2
    t += 0.0 if cfg["block_size"] == 128 else 0.1
    t += 0.0 if cfg["bank_capacity"] == 1 << 24 else 0.05
    t += 0.0 if cfg["primaries_per_wave"] == 1 << 20 else 0.03
    t += 0.0 if cfg["use_graph"] == 1 else 0.01
    return t * 1e-9


def test_coordinate_descent_finds_separable_optimum():
    best, t, trials = A.coordinate_descent(_cost)
    assert tuple(best["regs_variant"]) == (3, 3, 4, 4)
    assert best["block_size"] == 128 and best["bank_capacity"] == 1 << 24
    assert best["primaries_per_wave"] == 1 << 20 and best["use_graph"] == 1
    assert t == _cost(best)
    assert len(trials) <= sum(len(v) for v in A.SEARCH.values()) + 1


def test_cache_hit_skips_timing(tmp_path):
    p = W.config_water_open(n_histories=1000, npx=16, npy=16)
    calls = []

    def timer(cfg):
        calls.append(cfg)
        return _cost(cfg)

    path = tmp_path / "tune.json"
    e1 = A.autotune(p, path=path, timer=timer)
    n1 = len(calls)
    assert n1 > 1 and e1["block_size"] == 128
    e2 = A.autotune(p, path=path, timer=timer)
    assert len(calls) == n1 and e2 == json.loads(path.read_text())[next(iter(json.loads(path.read_text())))]
    assert A.overrides(e2)["regs_variant"] == [3, 3, 4, 4]
    # another workload shape is another key
    q = W.config_water_open(n_histories=1000, npx=32, npy=32)
    A.autotune(q, path=path, timer=timer)
    assert len(calls) > n1 and len(json.loads(path.read_text())) == 2
