"""Autotuner: accuracy rule for the map resolution (CPU) and the timed choice
of tile size and wave size with its JSON cache (GPU)."""
import json

import numpy as np
import pytest

from paper_1410_5780_gb300 import autotune as A, scenes as S


def test_accuracy_rule_texel_below_half_sample_spacing():
    for w in (S.make_tiny(), S.make_facade(), S.make_random_small(3)):
        R = A.accuracy_map_res(w, lo=64, hi=1 << 20)
        g = w.gen
        reach = float(np.max(g.cells_u * g.pitch) + np.max(g.cells_v * g.pitch))
        ext = float(np.ptp(g.origin, axis=0).max()) + 2 * reach
        spacing = float(np.min(g.pitch)) / w.n
        assert ext / (R - 2) <= 0.5 * spacing
        assert R == 64 or ext / (R // 2 - 2) > 0.5 * spacing  # the smallest such power of two
    assert A.accuracy_map_res(S.make_tracker()) == 8192  # capped


def test_size_class_is_stable():
    w = S.make_facade()
    assert A.size_class(w, 4096) == A.size_class(S.make_facade(), 4096)
    assert A.size_class(w, 4096) != A.size_class(w, 2048)


@pytest.mark.gpu
def test_autotune_picks_a_configuration_and_caches_it(tmp_path):
    w = S.make_facade(seed=9, n=4, map_res=1024, n_buildings=10, n_trees=4, n_poles=2, floors=2, per_floor=6,
                      target_tris=3000)
    cache = str(tmp_path / "tune.json")
    a = A.autotune(w, cache=cache, n_windows=2)
    assert a["tile"] in A.TILES and a["chunk_steps"] in A.WAVES and a["map_res"] == 1024
    assert a["bin_capacity"] >= 1 << 20 and not a["cached"]
    b = A.autotune(w, cache=cache)
    assert b["cached"] and b["tile"] == a["tile"] and b["chunk_steps"] == a["chunk_steps"]
    assert A.size_class(w, 1024) in json.load(open(cache))
