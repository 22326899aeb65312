#!/usr/bin/env python3
"""Benchmark of the GB300 shadow-sample path (3DPV method, arXiv 1410.5780).

Metric: shadow sample tests per second (lit sun steps x cell samples).  The
headline workload is the tracker plant, the largest single-GPU case: 500
two-axis trackers of 24 modules (6 x 12 cells, 4 x 4 samples per cell) on a
512 x 512 fractal terrain with 20 lattice pylons and a ridge (0.56 M
triangles), quarter-hour suns of a year at 40 N (17,519 daylight steps), an
8192^2 light window.  One bench step is one full-year evaluation; the timed
region runs the library's production path (each wave a replayed CUDA graph).
The BIPV facade (200 modules among buildings and trees, hourly year, 8 x 8
samples, 4096^2) is measured the same way and reported under "facade".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank evaluates its own seeded plant (independent
problems, weak scaling); the only collectives are the timing barrier and the
max-over-ranks of the timed region.  --impl reference times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "shadow sample tests/sec (sun steps x cell samples) at 1 GB300"
UNIT = "tests/s"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2

# algorithmic ALU work of the tile kernel (the roofline numerator).  The
# method's depth map must hold, at every texel a sample reads, the nearest of
# the triangles covering the texel centre: each such (texel, triangle)
# fragment costs 3 edge functions (2 FMA each) + barycentric depth (3 FMA) +
# key conversion and minimum (3) = 12 lane-ops; a sample test costs its
# position (2), projection to texel space and depth (6), floor/clamp/tile
# check (4), depth compare (2) = 14 lane-ops.
OPS_PER_TEXEL_WRITE = 12
OPS_PER_SAMPLE_TEST = 14


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tracker", choices=["facade", "tracker", "tiny"])
    ap.add_argument("--path", default="fused", choices=["fused", "map"])
    ap.add_argument("--chunk", type=int, default=0, help="sun steps per wave (0 = autotuned)")
    ap.add_argument("--tile", type=int, default=0, choices=[0, 32, 64, 128],
                    help="rasteriser tile side (0 = autotuned); with --chunk, the autotuner is skipped "
                         "(profiling runs pin the configuration the plain bench chose)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the batched, served and extension sections")
    ap.add_argument("--no-facade", action="store_true", help="skip the secondary facade measurement")
    ap.add_argument("--batch-scenes", type=int, default=256)
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--step-range", type=int, nargs=2, default=None, metavar=("BEGIN", "END"),
                    help="evaluate only sun steps [BEGIN, END) of the workload (profiling captures of one wave)")
    return ap.parse_args()


def make_workload(name: str, rank: int):
    from paper_1410_5780_gb300 import scenes as S
    if name == "facade":
        return S.make_facade(seed=1 + rank)
    if name == "tracker":
        return S.make_tracker(seed=2 + rank)
    return S.make_tiny()


def workload_config(w, name):
    return {"workload": {"facade": "BIPV facade: 200 modules on an 8-floor wall among 60 buildings, trees and "
                                   "poles (50k triangles), hourly year at 40 N",
                         "tracker": "tracker plant: 500 two-axis trackers of 24 modules on a 512 x 512 terrain with "
                                    "pylons and a ridge (0.56 M triangles), quarter-hour year",
                         "tiny": "tiny plain case: 2 modules, one 2 x 2 x 3 m box, 24 hourly steps of June 21"}[name],
            "modules": w.gen.n_modules, "cells": w.gen.n_cells, "samples_per_cell": w.n * w.n,
            "triangles": int(w.scene.n_tris), "sun_steps": int(w.sun.n_steps),
            "lit_steps": int((w.sun.xyz[:, 2] > 0).sum()), "map_res": w.map_res,
            "samples_per_step": w.samples_per_step}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons, n = [], [], set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                if int(parts[0]) != self.idx:
                    continue
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            n += 1
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": n}


# ---------------------------------------------------------------------------
# reference arm and CPU baseline: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
def oracle_sample_run(w, budget_s: float, chunk: int = 12, stride: int = 9):
    """Time the oracle (as it stands) on every `stride`-th lit step of the
    workload, chunk by chunk, until `budget_s` seconds of work are done."""
    import oracle
    lit = np.flatnonzero(w.sun.xyz[:, 2] > 0)[::stride]
    osc = oracle.OracleScene(w.scene.verts, w.scene.tris)
    threads = os.cpu_count() or 1
    done, t_tot = 0, 0.0
    for k in range(0, len(lit), chunk):
        steps = lit[k:k + chunk]
        t0 = time.perf_counter()
        oracle.evaluate_workload(w, steps=steps, want_mask=False, threads=threads, oscene=osc)
        t_tot += time.perf_counter() - t0
        done += len(steps)
        if t_tot >= budget_s:
            break
    tests = done * w.samples_per_step
    return tests / t_tot, threads, f"{done} of the {int((w.sun.xyz[:, 2] > 0).sum())} lit steps " \
        f"(every {stride}th), all {w.gen.n_modules} modules, {w.n}x{w.n} samples per cell, no parity mask; " \
        f"{t_tot:.1f} s", t_tot


def reduce_over_ranks(t_ms: float, tests: float, dist, device: str):
    """Whole-job timing of independent replicas: the slowest rank's time
    (every rank ran its own problem between the same barriers) and the tests
    of all ranks.  Without a process group, the local values."""
    if dist is None:
        return float(t_ms), float(tests)
    import torch
    dist.barrier()
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(tests)], dtype=torch.float64, device=device)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = make_workload(args.workload, 0)
    for _ in range(args.warmup):
        oracle_sample_run(w, budget_s=0.0, chunk=4)
    times, vals = [], []
    for _ in range(args.steps):
        v, cores, sample, t = oracle_sample_run(w, budget_s=8.0, chunk=6)
        vals.append(v)
        times.append(t)
    value = float(statistics.mean(vals))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(statistics.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": workload_config(w, args.workload),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def code_digest(path: str) -> str:
    """sha256 of a CUDA/C source with its comments and whitespace removed: the
    digest changes with the code, not with its comments."""
    import hashlib
    import re
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return hashlib.sha256(re.sub(r"\s+", "", text).encode()).hexdigest()


def profiled_traffic(workload: str, tile: int, kernel: str = "k_tile_warp"):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary
    (profiles/<kernel>_<workload>*.md), if it was taken on the current code of
    kernels.cu with the same tile side (else None)."""
    import glob
    import re
    src = os.path.join(ROOT, "paper_1410_5780_gb300", "csrc", "kernels.cu")
    try:
        digest = code_digest(src)
    except OSError:
        return None
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_{workload}*.md"))):
        try:
            rec = json.loads(re.search(r"<!-- traffic: (\{.*?\}) -->", open(path).read()).group(1))
        except (OSError, AttributeError, ValueError):
            continue
        if rec.get("code_sha256") == digest and rec.get("tile") == tile and rec.get("kernel", kernel) == kernel:
            return rec["bytes_per_launch"]
    return None


def input_bytes(w) -> int:
    m = w.gen.n_modules
    b = w.scene.verts.nbytes + w.scene.tris.nbytes + 64 * m
    b += sum(4 * len(l.cell_sub) for l in w.gen.layouts) + w.gen.pivots.nbytes
    b += w.sun.xyz.nbytes + w.sun.dni.nbytes + w.sun.dhi.nbytes + w.sun.dt_h.nbytes
    if w.poses is not None:
        b += w.poses.nbytes
    return int(b)


def _batched_vs_plain(dev: int, ws, depth_format: int = 0) -> dict:
    import torch
    from paper_1410_5780_gb300 import pv3d
    tests = sum(w.n_tests() for w in ws)
    with pv3d.Context(device=dev, depth_format=depth_format) as ctx:
        gids = [pv3d.load_workload(ctx, w) for w in ws]
        ns = [w.n for w in ws]
        rs = [w.map_res for w in ws]
        ctx.evaluate_batch(gids[:8], n=ns[:8], map_res=rs[:8])  # warm-up
        for w, g in zip(ws[:4], gids[:4]):
            ctx.evaluate(g, n=w.n, map_res=w.map_res)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plain = [ctx.evaluate(g, n=w.n, map_res=w.map_res) for w, g in zip(ws, gids)]
        torch.cuda.synchronize()
        t_plain = time.perf_counter() - t0
        t0 = time.perf_counter()
        batch = ctx.evaluate_batch(gids, n=ns, map_res=rs)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        same = all(bool(torch.equal(a["energy"], b["energy"])) for a, b in zip(plain, batch))
        loss = [100.0 * (1.0 - float(b["energy"].double().sum()) / max(float(b["energy_unshaded"].double().sum()), 1e-30))
                for b in batch]
    return {"tests": int(tests), "plain_tests_per_s": tests / t_plain, "batched_tests_per_s": tests / t_batch,
            "speedup": t_plain / t_batch, "batched_equals_plain": same, "plain_s": t_plain, "batched_s": t_batch,
            "_loss": loss}


def batched_section(dev: int, n_scenes: int) -> dict:
    """Batched scenes of uneven size (log-uniform triangles and modules,
    latitudes 0-60 deg, 100-4400 sun steps): the plain per-scene loop against
    one batched call (all scenes' sun steps packed into shared waves), with
    FP32 depth and with 24-bit fixed-point depth; also a mix of small scenes,
    where one scene alone does not fill the GPU."""
    from paper_1410_5780_gb300 import pv3d, scenes as S
    ws = S.make_batch(seed=4, n_scenes=n_scenes)
    mix = _batched_vs_plain(dev, ws)
    u24 = _batched_vs_plain(dev, ws, depth_format=pv3d.PV3D_DEPTH_U24)
    dl = np.abs(np.array(u24.pop("_loss")) - np.array(mix.pop("_loss")))
    mix["workload"] = (f"{n_scenes} scenes: triangles log-uniform 1e3-2e5, modules log-uniform 10-2000, "
                       "latitude U(0,60), 100-4400 hourly sun steps, 4x4 samples, map 512-4096")
    mix["depth_u24"] = {"plain_tests_per_s": u24["plain_tests_per_s"], "batched_tests_per_s": u24["batched_tests_per_s"],
                        "speedup": u24["speedup"], "batched_equals_plain": u24["batched_equals_plain"],
                        "loss_pp_vs_f32": {"max_abs": float(dl.max()), "mean_abs": float(dl.mean())}}
    small = _batched_vs_plain(dev, S.make_batch(seed=6, n_scenes=n_scenes, tris=(1e3, 2e4), mods=(10, 100),
                                                steps=(100, 400)))
    small.pop("_loss")
    small["workload"] = f"{n_scenes} small scenes: 1e3-2e4 triangles, 10-100 modules, 100-400 sun steps"
    mix["small_scenes"] = small
    mix["clock"] = "host wall clock around each form, device synchronised"
    return mix


def extensions_section(ctx, gid, w, stream) -> dict:
    """The model extensions on the bench workload (device time of one
    full-year evaluation each, CUDA events on the evaluation's stream): series
    strings of 5 modules along each floor, one 1024-texel light window per
    string (window groups), the azimuth-zenith sky map (36 x 9 bins), diffuse
    shading (sky view over 9 x 36 patches, then a year with the diffuse term
    shaded), and the clear-sky sun table made on the device."""
    import torch
    from paper_1410_5780_gb300 import pv3d

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        a.record(stream)
        r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), r

    base, r0 = timed(lambda: ctx.evaluate(gid, n=w.n, map_res=w.map_res, outputs=("energy",),
                                          stream=stream.cuda_stream))
    out = {"plain_ms": base, "tests": r0["tests"]}
    # FP32 Kahan yearly energy sums against the FP64 sum of the same per-step powers
    rk = ctx.evaluate(gid, n=w.n, map_res=w.map_res, outputs=("energy", "power"), stream=stream.cuda_stream)
    torch.cuda.synchronize()
    p64 = rk["power"].double().cpu().numpy()
    e64 = (p64 * w.sun.dt_h.astype(np.float64)[:, None]).sum(0)
    ek = rk["energy"].cpu().numpy()
    rel = np.abs(ek - e64) / np.maximum(np.abs(e64), 1e-30)
    out["kahan_fp32_vs_fp64"] = {"max_rel_err": float(rel.max()), "mean_rel_err": float(rel.mean()),
                                 "modules": int(len(ek)), "steps": int(w.sun.n_steps)}
    gen = w.gen
    sid = ctx.scene_load(w.scene.verts, w.scene.tris)
    saved = gen.string.copy()
    gen.string = (np.arange(gen.n_modules) // 5).astype(np.int32)
    g2 = ctx.generator_define(sid, gen)
    gen.string = saved
    ctx.set_sun(g2, w.sun.xyz, w.sun.dni, w.sun.dhi, w.sun.dt_h)
    t, r = timed(lambda: ctx.evaluate(g2, n=w.n, map_res=w.map_res, stream=stream.cuda_stream,
                                      outputs=("energy", "string_energy", "string_energy_unshaded")))
    se, seu = r["string_energy"].double().sum().item(), r["string_energy_unshaded"].double().sum().item()
    out["strings"] = {"ms": t, "strings": int(len(np.unique(np.arange(gen.n_modules) // 5))),
                      "loss_pct": 100.0 * (1.0 - se / seu)}
    t, r = timed(lambda: ctx.evaluate(g2, n=w.n, map_res=1024, stream=stream.cuda_stream,
                                      outputs=("energy", "energy_unshaded"),
                                      window_groups=pv3d.PV3D_WINDOWS_PER_STRING))
    e, eu = r["energy"].double().sum().item(), r["energy_unshaded"].double().sum().item()
    out["windows_per_string"] = {"ms": t, "windows": out["strings"]["strings"], "map_res": 1024,
                                 "waves": int(r["waves"]), "loss_pct": 100.0 * (1.0 - e / eu)}
    t, r = timed(lambda: ctx.evaluate(g2, n=w.n, map_res=w.map_res, stream=stream.cuda_stream,
                                      outputs=("energy",), heat_bins=(36, 9)))
    out["sky_map"] = {"ms": t, "bins": [36, 9], "occupied_bins": int((r["heat_steps"] > 0).sum().item())}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f = ctx.sky_view(g2, rings=9, sectors=36, n=w.n, map_res=w.map_res)
    t_sky = (time.perf_counter() - t0) * 1e3
    t, r = timed(lambda: ctx.evaluate(g2, n=w.n, map_res=w.map_res, stream=stream.cuda_stream,
                                      outputs=("energy", "energy_unshaded"), diffuse_shading=True))
    e, eu = r["energy"].double().sum().item(), r["energy_unshaded"].double().sum().item()
    out["diffuse"] = {"sky_view_ms_wall": t_sky, "patches": 324, "mean_cell_fraction": float(f.mean()),
                      "year_ms": t, "loss_pct_with_diffuse": 100.0 * (1.0 - e / eu)}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n = ctx.set_sun_clear_sky(g2, 40.0, 1.0, day_first=1, n_days=365)
    out["sun_table"] = {"ms_wall": (time.perf_counter() - t0) * 1e3, "steps": int(n),
                        "what": "hourly clear-sky year at 40 N, daylight steps kept"}
    ctx.release(g2)
    ctx.release(sid)
    return out


def tracker_windows_section(ctx, gid, w, stream, n_steps: int = 1024) -> dict:
    """One light window per tracker on the tracker plant, on a bounded sample
    (the first ``n_steps`` quarter-hour steps, device time): the plant-wide
    window at the workload's resolution against per-tracker windows of 256 and
    512 texels (every tracker's table still shades the others)."""
    import torch
    from paper_1410_5780_gb300 import pv3d

    out = {"steps": n_steps, "trackers": int(w.gen.pivots.shape[0])}
    for name, res, mode in (("plant_window", w.map_res, pv3d.PV3D_WINDOWS_ONE),
                            ("per_tracker_256", 256, pv3d.PV3D_WINDOWS_PER_TRACKER),
                            ("per_tracker_512", 512, pv3d.PV3D_WINDOWS_PER_TRACKER)):
        def run():
            return ctx.evaluate(gid, n=w.n, map_res=res, step_end=n_steps, stream=stream.cuda_stream,
                                outputs=("energy", "energy_unshaded"), window_groups=mode)
        run()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = run()
        b.record(stream)
        torch.cuda.synchronize()
        e, eu = r["energy"].double().sum().item(), r["energy_unshaded"].double().sum().item()
        out[name] = {"map_res": res, "ms": a.elapsed_time(b), "tests_per_s": r["tests"] / (a.elapsed_time(b) * 1e-3),
                     "waves": int(r["waves"]), "loss_pct": 100.0 * (1.0 - e / eu)}
    return out


def serving_section(dev: int, n_requests: int) -> dict:
    """Served evaluation of a stream of requests over a pool of resident
    scenes (1e3-5.2e5 triangles, 10-2000 modules), each request a random
    range of 100-4400 sun steps of its scene.  Three runs over the same
    request list: the plain per-scene loop (one synchronous evaluation after
    another), the served capacity (every request submitted at once:
    continuous batching into shared waves), and Poisson arrivals at 80 % of
    that capacity, with p50/p99 submit-to-result latency."""
    import torch
    from paper_1410_5780_gb300 import pv3d, scenes as S
    rng = np.random.default_rng(11)
    pool = S.make_batch(seed=5, n_scenes=24, tris=(1e3, 5.2e5))
    with pv3d.Context(device=dev, hbm_budget_bytes=120 << 30) as ctx:
        gids = [pv3d.load_workload(ctx, w) for w in pool]
        reqs = []
        for _ in range(n_requests):
            q = int(rng.integers(len(pool)))
            w = pool[q]
            k = int(rng.integers(min(100, w.sun.n_steps), w.sun.n_steps + 1))
            b = int(rng.integers(0, w.sun.n_steps - k + 1))
            lit = int((w.sun.xyz[b:b + k, 2] > 0).sum())
            reqs.append((q, b, b + k, lit * w.samples_per_step))
        total_tests = sum(r[3] for r in reqs)

        def submit(q, b, e):
            w = pool[q]
            return ctx.submit(gids[q], n=w.n, map_res=w.map_res, step_begin=b, step_end=e)

        for q in range(min(4, len(pool))):  # warm-up
            assert ctx.poll(submit(q, 0, 100)[0], timeout_ms=-1) == pv3d.PV3D_OK
            ctx.evaluate(gids[q], n=pool[q].n, map_res=pool[q].map_res, step_end=100)
        # plain per-scene loop over the same requests
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for q, b, e, _ in reqs:
            w = pool[q]
            ctx.evaluate(gids[q], n=w.n, map_res=w.map_res, step_begin=b, step_end=e)
        torch.cuda.synchronize()
        t_plain = time.perf_counter() - t0
        # capacity: every request at once
        t0 = time.perf_counter()
        ids = [submit(q, b, e)[0] for q, b, e, _ in reqs]
        for rid in ids:
            assert ctx.poll(rid, timeout_ms=-1) == pv3d.PV3D_OK
        t_cap = time.perf_counter() - t0
        capacity_rps = n_requests / t_cap
        # Poisson arrivals at 80 % of the capacity
        rate = 0.8 * capacity_rps
        gaps = rng.exponential(1.0 / rate, n_requests)
        t0 = time.perf_counter()
        t_arr = t0 + np.cumsum(gaps)
        live, lat, lat_tests = {}, [], []
        for i, (q, b, e, nt) in enumerate(reqs):
            while time.perf_counter() < t_arr[i]:
                for rid in list(live):
                    if ctx.poll(rid, timeout_ms=0) == pv3d.PV3D_OK:
                        arr, n_t = live.pop(rid)
                        lat.append(arr["latency_ms"])
                        lat_tests.append(n_t)
                time.sleep(0.0002)
            rid, arrays = submit(q, b, e)
            live[rid] = (arrays, nt)
        for rid in list(live):
            assert ctx.poll(rid, timeout_ms=-1) == pv3d.PV3D_OK
            arr, n_t = live.pop(rid)
            lat.append(arr["latency_ms"])
            lat_tests.append(n_t)
        span = time.perf_counter() - t0
    lat = np.array(lat)
    lat_tests = np.array(lat_tests, float)
    small = lat_tests <= np.percentile(lat_tests, 50)
    return {"workload": f"{n_requests} requests over {len(pool)} resident scenes (1e3-5.2e5 triangles, 10-2000 "
                        "modules), each a random range of 100-4400 hourly sun steps; the same list for all three runs",
            "tests": int(total_tests),
            "plain_tests_per_s": total_tests / t_plain, "plain_s": t_plain,
            "served_capacity_tests_per_s": total_tests / t_cap, "served_capacity_s": t_cap,
            "served_vs_plain": t_plain / t_cap,
            "capacity_requests_per_s": capacity_rps, "arrival_rate_per_s": rate,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "p50_ms_smaller_half": float(np.percentile(lat[small], 50)),
            "p99_ms_smaller_half": float(np.percentile(lat[small], 99)),
            "poisson_tests_per_s": total_tests / span, "requests": n_requests,
            "clock": "host wall clock; latency from pv3d_submit to the result (the library's own stamp)"}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tile_kernel_rooflines(work, stages_ms, tile, n_waves, hbm_gbs, alu_tops, raster_peak, workload):
    """Roofline figures of the two tile kernels per launch (one launch a wave).

    Algorithmic work per launch, from the work counters of one evaluation:
    * bytes (the HBM byte model of a depth-map design restricted to the
      kernel's tiles): 4 B per texel of every tile it takes (the depth tile
      written once) + 4 B per sample it tests (the texel gather);
    * lane-ops: 12 per fragment (a kept triangle covering a texel a sample
      reads: 3 edge functions, barycentric depth, key and minimum) + 14 per
      sample test (position, projection, texel, compare);
    * fragments F (k_raster_test: depth atomicMin writes into the shared tile).
    """
    nw = max(n_waves, 1)
    heavy = {"tiles": work["heavy_tiles"], "samples": work["heavy_sample_tests"],
             "fragments": work["heavy_texel_writes"], "ms": stages_ms["heavy"]}
    warp = {"tiles": work["nonempty_tiles"] - work["heavy_tiles"],
            "samples": work["sample_tests"] - work["heavy_sample_tests"],
            "fragments": work["texel_writes"] - work["heavy_texel_writes"], "ms": stages_ms["raster"]}
    out = {}
    for name, k in (("k_tile_warp", warp), ("k_raster_test", heavy)):
        launch_ms = k["ms"] / nw
        t = max(launch_ms * 1e-3, 1e-12)
        byts = (4.0 * tile * tile * k["tiles"] + 4.0 * k["samples"]) / nw
        ops = (OPS_PER_TEXEL_WRITE * k["fragments"] + OPS_PER_SAMPLE_TEST * k["samples"]) / nw
        gbs = byts / t / 1e9
        tops = ops / t / 1e12
        d = {"avg_launch_ms": launch_ms, "ms_per_step": k["ms"],
             "per_launch": {"tiles": k["tiles"] / nw, "sample_tests": k["samples"] / nw,
                            "fragments": k["fragments"] / nw, "algorithmic_bytes": byts, "lane_ops": ops},
             "hbm": {"achieved": gbs, "peak": hbm_gbs, "unit": "GB/s", "frac": gbs / hbm_gbs},
             "alu": {"achieved": tops, "peak": alu_tops, "unit": "T lane-ops/s", "frac": tops / alu_tops},
             "traffic": profiled_traffic(workload, tile, name)}
        if name == "k_raster_test" and raster_peak:
            fr = k["fragments"] / nw / t / 1e9
            d["raster"] = {"achieved": fr, "peak": raster_peak, "unit": "G atomicMin/s", "frac": fr / raster_peak}
        out[name] = d
    return out


def path_byte_model(w, work, tile, chunk, n_steps_lit, t_ms_per_step):
    """The hot path's algorithmic bytes per sun step (HBM byte model of a
    depth-map design): 4 R2_occ (occupied-tile texels, written once) + 4 S
    (one texel gathered per sample) + 36 T / K (triangles read once per wave
    of K steps) + outputs (1 B per cell, 12 B per module)."""
    r2_occ = work["nonempty_tiles"] * tile * tile / max(n_steps_lit, 1)
    S = w.samples_per_step
    T = int(w.scene.n_tris) + 2 * w.gen.n_modules
    b_step = 4.0 * r2_occ + 4.0 * S + 36.0 * T / chunk + w.gen.n_cells + 12.0 * w.gen.n_modules
    achieved = b_step * n_steps_lit / (t_ms_per_step * 1e-3) / 1e9
    return {"R2_occ_per_step": r2_occ, "S": S, "T": T, "K": chunk, "bytes_per_step": b_step,
            "achieved_GBps": achieved}


def measure(args, name, dev, dist, rank, world, steps, warmup, tile=0, chunk=0):
    """Time ``steps`` full evaluations of workload ``name`` on the production
    path; returns the line's fields for it (rank 0) and the objects for the
    e2e and extension sections."""
    import torch
    from paper_1410_5780_gb300 import autotune, pv3d
    w = make_workload(name, rank)
    path = pv3d.PV3D_PATH_FUSED if args.path == "fused" else pv3d.PV3D_PATH_MAP
    # tile size, sun steps per wave and bin pool from the autotuner (short
    # timed trials, not part of the timed region); the map resolution is the
    # workload's own
    if tile and chunk:
        tuned = {"tile": tile, "chunk_steps": chunk, "bin_capacity": 0}  # 0: the library's pool
    else:
        tuned = autotune.autotune(w, device=dev, cache=None, n_windows=6)
        tuned["tile"] = tile or tuned["tile"]
    chunk = chunk or tuned["chunk_steps"]
    ctx = pv3d.Context(device=dev, map_res=w.map_res, chunk_steps=chunk, tile=tuned["tile"],
                       bin_capacity=tuned["bin_capacity"])
    gid = pv3d.load_workload(ctx, w)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=f"cuda:{dev}")
    sb, se = args.step_range or (0, 0)

    def evaluate(profile=0):
        return ctx.evaluate(gid, n=w.n, map_res=w.map_res, outputs=("energy", "energy_unshaded"),
                            stream=stream.cuda_stream, path=path, profile=profile, step_begin=sb, step_end=se)

    for _ in range(max(warmup, 0)):
        evaluate()
    torch.cuda.synchronize()
    # timed region: K evaluations on the production path (waves replayed from
    # one captured CUDA graph), L2 flushed between them outside the events
    sampler = ClockSampler(dev)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    tests = launches = 0
    results = []
    torch.cuda.nvtx.range_push("timed")
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        r = evaluate(profile=0)
        ev[k][1].record(stream)
        tests += r["tests"]
        launches += r["kernel_launches"]
        results.append(r)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    t_ms, tests_all = reduce_over_ranks(t_ms, tests, dist, f"cuda:{dev}")
    value = tests_all / (t_ms * 1e-3)
    # untimed: the stage split (per-kernel launches with stage events) and
    # the work counters (a counting run) of the same evaluation
    torch.cuda.synchronize()
    evaluate(profile=1)
    prof = ctx.last_profile()
    evaluate(profile=3)
    work = ctx.last_profile()
    e_loss = 100.0 * (1.0 - float(results[-1]["energy"].sum()) / float(results[-1]["energy_unshaded"].sum()))
    out = {"w": w, "ctx": ctx, "gid": gid, "stream": stream, "path": path, "tuned": tuned, "chunk": chunk}
    if rank != 0:
        return out
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    props = torch.cuda.get_device_properties(dev)
    alu_peak = props.multi_processor_count * 128 * sm_max * 1e6 / 1e12  # T lane-ops/s
    stages = {s_: float(prof[f"{s_}_ms"]) for s_ in pv3d.STAGES}
    raster_peak = None
    try:
        raster_peak = pv3d.raster_peak(dev)["g_atomics_per_s"]
    except (AttributeError, pv3d.PV3DError, OSError):
        raster_peak = None
    kern = tile_kernel_rooflines(work, stages, tuned["tile"], prof["waves"], hbm, alu_peak, raster_peak, name)
    dom = max(kern, key=lambda k: kern[k]["ms_per_step"])
    kd = kern[dom]
    lit = int(results[-1]["steps_lit"])
    t_step = t_ms / steps
    model = path_byte_model(w, work, tuned["tile"], chunk, lit, t_step / max(world, 1) * max(world, 1))
    model["frac"] = model["achieved_GBps"] / hbm
    out["line"] = {
        "value": value, "ms_per_step": t_step, "steps": steps, "warmup": warmup,
        "config": dict(workload_config(w, name), path=args.path, l2="flushed between steps (512 MB write)",
                       waves_per_step=int(prof["waves"]), annual_loss_pct=round(e_loss, 4),
                       timed_path="production: each wave a replayed CUDA graph, no stage events",
                       autotuned={"tile": tuned["tile"], "chunk_steps": chunk, "bin_capacity": tuned["bin_capacity"]}),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": kd["hbm"]["achieved"], "peak": hbm, "unit": "GB/s",
                     "frac": kd["hbm"]["frac"], "traffic": kd["traffic"],
                     "peak_source": "hbm_gbs of MEASURED_PEAKS.json (measured copy bandwidth)",
                     "algorithmic": "4 B per texel of each tile the kernel takes (depth tile written once) + 4 B per "
                                    "sample it tests (texel gather), per launch (one wave), over its average launch "
                                    "time (stage events of an untimed run of the same evaluation)",
                     "traffic_source": f"DRAM read+write bytes of one launch, ncu capture in profiles/{dom}_{name}*.md "
                                       "taken with the same tile side (null if the code of kernels.cu changed since)",
                     "alu": kd["alu"], "per_launch": kd["per_launch"], "avg_launch_ms": kd["avg_launch_ms"],
                     "alu_peak_source": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {sm_max:.0f} MHz",
                     "kernels": kern, "path_byte_model": model},
        "work_per_step": {"sample_tests_in_tested_tiles": work["sample_tests"] / max(lit, 1),
                          "fragments": work["texel_writes"] / max(lit, 1),
                          "nonempty_tiles": work["nonempty_tiles"] / max(lit, 1),
                          "heavy_tiles": work["heavy_tiles"] / max(lit, 1),
                          "heavy_why_per_year": {"receivers": work["heavy_why"][0], "binned": work["heavy_why"][1],
                                                 "kept": work["heavy_why"][2]},
                          "binned_pairs": work["binned_tris"] / max(lit, 1),
                          "pair_tests": work["pair_tests"] / max(lit, 1)},
        "stages_ms_per_step": stages,
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    return out


def e2e_section(m, args, world):
    """The same metric through the C ABI with host arrays: scene, generator,
    sun (and poses) uploaded from host memory, the evaluation with host
    outputs, the energies read back -- every step."""
    import torch
    from paper_1410_5780_gb300 import pv3d
    w, ctx = m["w"], m["ctx"]
    h2d = input_bytes(w)
    d2h = 16 * w.gen.n_modules
    t_e2e = []
    r2 = None
    for k in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g2 = pv3d.load_workload(ctx, w)
        r2 = ctx.evaluate(g2, n=w.n, map_res=w.map_res, outputs=("energy", "energy_unshaded"), device=False,
                          path=m["path"])
        ctx.release(g2)
        t_e2e.append(time.perf_counter() - t0)
    e2e_val = r2["tests"] / statistics.mean(t_e2e)
    return {"value": e2e_val * world, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "includes": "scene/generator/sun/pose upload from host arrays, evaluation, host read-back of the "
                        "energies (best of the library's pools, host wall clock)"}


def run_ours(args, rank, world, dist):
    import torch
    from paper_1410_5780_gb300 import pv3d
    pv3d.load(build_if_missing=True)
    local = int(os.environ.get("LOCAL_RANK", rank))
    dev = local if torch.cuda.device_count() > local else 0
    torch.cuda.set_device(dev)
    m = measure(args, args.workload, dev, dist, rank, world, args.steps, args.warmup, args.tile, args.chunk)
    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": m["line"]["value"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["line"]["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic"}
        line.update({k: v for k, v in m["line"].items() if k not in ("value", "ms_per_step", "steps", "warmup")})
    if not args.no_e2e:
        e2e = e2e_section(m, args, world)
        if rank == 0:
            line["e2e"] = e2e
    if rank == 0 and not args.no_serving and args.workload == "tracker":
        line["extensions"] = tracker_windows_section(m["ctx"], m["gid"], m["w"], m["stream"])
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample, _ = oracle_sample_run(m["w"], budget_s=15.0)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    m["ctx"].close()
    # the facade (the secondary workload): the same measurement, its own line fields
    if args.workload != "facade" and not args.no_facade and args.step_range is None:
        f = measure(args, "facade", dev, dist, rank, world, max(3, args.steps), max(3, args.warmup))
        if rank == 0:
            line["facade"] = f["line"]
            if not args.no_serving:
                line["facade"]["extensions"] = extensions_section(f["ctx"], f["gid"], f["w"], f["stream"])
        f["ctx"].close()
    if rank == 0 and not args.no_serving and world == 1:
        line["batched"] = batched_section(dev, args.batch_scenes)
        line["serving"] = serving_section(dev, args.requests)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
        tdist.init_process_group(backend=backend)
        dist = tdist
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
