"""Autotuner for the shadow-sample path: rasteriser tile size, sun steps per
wave, initial bin-pool capacity and (optionally) shadow-map resolution.

* Map resolution is an accuracy choice, not a speed one: when asked (``map_res=0``)
  it is the smallest power of two whose texel is at most half the sample
  spacing over the generator's extent, within [512, 8192].
* Tile side (32, 64 or 128 texels) and wave size K (32..256 sun steps) are chosen by
  timing short trial evaluations through the C ABI on step windows spread over
  the sun table; the candidates within ``FINAL_MARGIN`` of the fastest trial are
  then timed over the whole sun table (best of two, while that stays within
  ``FINAL_BUDGET_MS`` of device time), and the fastest per-step device time wins.
* The bin pool is pre-sized from the trials' largest per-wave demand, so the
  full run does not have to grow it (and rerun) on overflow.

Choices are cached in a JSON file keyed by a scene-size class (triangles,
modules, cells and samples per step rounded to powers of two, map resolution).
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import pv3d

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "pv3d", "autotune.json")
TILES = (32, 64, 128)
WAVES = (32, 64, 128, 256)
FINAL_MARGIN = 1.15       # trial candidates this close to the fastest are re-timed
FINAL_BUDGET_MS = 20000.0  # device time the whole-table re-timing may spend


def accuracy_map_res(w, lo: int = 512, hi: int = 8192) -> int:
    """Smallest power of two R with texel <= half the sample spacing."""
    g = w.gen
    pts = g.pivots if g.pivots.shape[0] else g.origin
    reach = float(np.max(g.cells_u * g.pitch) + np.max(g.cells_v * g.pitch))
    extent = float(np.ptp(pts, axis=0).max()) + 2.0 * reach
    spacing = float(np.min(g.pitch)) / w.n
    r = lo
    while r < hi and extent / (r - 2) > 0.5 * spacing:
        r *= 2
    return r


def size_class(w, map_res: int) -> str:
    def p2(x):
        return int(2 ** round(math.log2(max(x, 1))))
    return f"t{p2(w.scene.n_tris)}_m{p2(w.gen.n_modules)}_s{p2(w.samples_per_step)}_r{map_res}_n{w.n}"


def _windows(n_steps: int, k: int, n_win: int):
    k = min(k, n_steps)
    starts = np.linspace(0, max(n_steps - k, 0), n_win).astype(int)
    return [(int(b), int(b + k)) for b in starts]


def autotune(w, device: int = 0, map_res: int | None = None, cache: str | None = DEFAULT_CACHE,
             n_windows: int = 3, verbose: bool = False) -> dict:
    """Return {"tile", "chunk_steps", "map_res", "bin_capacity", "trial_ms_per_step"} for workload ``w``."""
    import torch
    R = int(w.map_res if map_res is None else (map_res or accuracy_map_res(w)))
    key = size_class(w, R)
    table = {}
    if cache and os.path.exists(cache):
        try:
            with open(cache) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
        if key in table:
            return dict(table[key], cached=True)
    best = None
    demand = 0
    trials = []
    for tile in TILES:
        with pv3d.Context(device=device, tile=tile, map_res=R) as ctx:
            gid = pv3d.load_workload(ctx, w)
            for k in WAVES:
                wins = _windows(w.sun.n_steps, k, n_windows)
                ctx.evaluate(gid, n=w.n, map_res=R, step_begin=wins[0][0], step_end=wins[0][1], chunk_steps=k)
                torch.cuda.synchronize()
                ms, steps = 0.0, 0
                for b, e in wins:
                    r = ctx.evaluate(gid, n=w.n, map_res=R, step_begin=b, step_end=e, chunk_steps=k)
                    ms += r["device_ms"]
                    steps += e - b
                    demand = max(demand, int(r["binned_tris"] / max(r["waves"], 1)))
                per_step = ms / max(steps, 1)
                if verbose:
                    print(f"autotune {key}: tile {tile} K {k}: {per_step:.4f} ms/step")
                trials.append((per_step, tile, k))
                if best is None or per_step < best["trial_ms_per_step"]:
                    best = {"tile": tile, "chunk_steps": k, "map_res": R, "trial_ms_per_step": per_step}
    # trial windows cover part of the year: re-time the close candidates on all of it
    trials.sort()
    finalists = [(t, k) for ms, t, k in trials if ms <= FINAL_MARGIN * trials[0][0]]
    n = w.sun.n_steps
    if len(finalists) > 1 and 2 * len(finalists) * n * trials[0][0] <= FINAL_BUDGET_MS:
        final = None
        for tile in sorted({t for t, _ in finalists}):
            with pv3d.Context(device=device, tile=tile, map_res=R,
                              bin_capacity=int(max(demand * 1.25, 1 << 20))) as ctx:
                gid = pv3d.load_workload(ctx, w)
                for t, k in finalists:
                    if t != tile:
                        continue
                    ms = min(ctx.evaluate(gid, n=w.n, map_res=R, chunk_steps=k)["device_ms"] for _ in range(2))
                    if verbose:
                        print(f"autotune {key}: tile {tile} K {k}: {ms / n:.4f} ms/step over all {n} steps")
                    if final is None or ms < final[0]:
                        final = (ms, tile, k)
        best.update(tile=final[1], chunk_steps=final[2], final_ms_per_step=final[0] / n)
    best["bin_capacity"] = int(max(demand * 1.25, 1 << 20))
    best["when"] = time.strftime("%Y-%m-%dT%H:%M:%S")
    if cache:
        table[key] = best
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = cache + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, cache)
    return dict(best, cached=False)
