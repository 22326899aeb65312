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


class _FakeCtx:
    """Stands in for pv3d.Context: per-step device times by tile size, one
    set for the trial windows and another for whole-table runs."""
    trial = {32: 2.0, 64: 1.05, 128: 1.0}
    whole = {32: 2.0, 64: 1.05, 128: 1.2}
    whole_calls = []

    def __init__(self, device=0, tile=64, map_res=0, bin_capacity=0):
        self.tile = tile

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def evaluate(self, gid, n=3, map_res=0, step_begin=0, step_end=0, chunk_steps=0):
        steps = (step_end or self.n_steps) - step_begin
        if step_begin == 0 and step_end == 0:
            _FakeCtx.whole_calls.append((self.tile, chunk_steps))
            per = self.whole[self.tile]
        else:
            per = self.trial[self.tile]
        return {"device_ms": per * steps * (1.0 if chunk_steps == 256 else 1.01), "binned_tris": 1000, "waves": 1}


def _fake_tune(monkeypatch, budget_ms):
    import torch
    w = S.make_tiny()
    _FakeCtx.n_steps = w.sun.n_steps
    _FakeCtx.whole_calls = []
    monkeypatch.setattr(A.pv3d, "Context", _FakeCtx)
    monkeypatch.setattr(A.pv3d, "load_workload", lambda ctx, w: 1)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(A, "FINAL_BUDGET_MS", budget_ms)
    return A.autotune(w, cache=None, n_windows=2)


def test_autotune_whole_table_decides_between_close_trials(monkeypatch):
    """Tile 128 wins the trial windows, tile 64 (within the margin) the whole
    table: the whole-table re-timing picks 64; tile 32 (twice as slow) is not
    re-timed."""
    a = _fake_tune(monkeypatch, 1e9)
    assert a["tile"] == 64 and a["chunk_steps"] == 256
    assert {t for t, _ in _FakeCtx.whole_calls} == {64, 128}
    assert a["final_ms_per_step"] == pytest.approx(1.05)


def test_autotune_trials_decide_when_the_table_is_too_long(monkeypatch):
    """Past the device-time budget the trial windows alone decide."""
    a = _fake_tune(monkeypatch, 0.0)
    assert a["tile"] == 128 and not _FakeCtx.whole_calls and "final_ms_per_step" not in a
