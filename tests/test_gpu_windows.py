"""GPU parity of light windows per window group (one per tracker, string or
inverter input) against the FP64 oracle.

The oracle's exact ray test does not depend on the light windows; its parity
mask (rays within one texel of an edge) is taken at the texel of the
generator-wide window, which is coarser than every group's window here, so the
mask stays conservative.
"""
import numpy as np
import pytest

import oracle
from paper_1410_5780_gb300 import pv3d, scenes as S

from parity import FLAG_AGREEMENT, compare, energy_checks, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    pv3d.load(build_if_missing=True)
    c = pv3d.Context(device=0)
    yield c
    c.close()


def mini_tracker():
    return S.make_tracker(seed=9, n=4, map_res=1024, grid=(4, 3), terrain_n=64, spacing=1.5, n_pylons=2,
                          step_h=1.0, days=np.array([30, 172, 300]))


def mini_facade():
    return S.make_facade(seed=7, n=4, map_res=1024, n_buildings=12, n_trees=6, n_poles=4, floors=2, per_floor=6,
                         target_tris=4000, days=np.array([20, 110, 200, 300]), radius=80.0)


def check(ctx, w, mode, map_res, chunk_steps=0):
    gid = pv3d.load_workload(ctx, w)
    g = run_gpu(ctx, gid, w, window_groups=mode, map_res=map_res, chunk_steps=chunk_steps)
    o = oracle.evaluate_workload(w)
    steps = np.arange(w.sun.n_steps)
    st = compare(w, g, o, steps)
    assert st["agree"] >= FLAG_AGREEMENT, st
    assert st["cell_ok"] == 1.0, st
    energy_checks(w, g, o, steps)
    assert g["tests"] == int((w.sun.xyz[:, 2] > 0).sum()) * w.samples_per_step
    ctx.release(gid)
    return g, o


def test_window_per_tracker(ctx):
    """12 trackers, each its own 512-texel window (finer than the plant's
    1024-texel window); the other trackers' tables shade each one."""
    w = mini_tracker()
    g, o = check(ctx, w, pv3d.PV3D_WINDOWS_PER_TRACKER, 512, chunk_steps=7)
    assert o["counts"].sum() > 0  # trackers do shade one another


def test_window_per_string_facade(ctx):
    """Facade modules in strings of 3, one 256-texel window per string."""
    w = mini_facade()
    w.gen.string = (np.arange(w.gen.n_modules) // 3).astype(np.int32)
    check(ctx, w, pv3d.PV3D_WINDOWS_PER_STRING, 256)


def test_one_group_is_the_plain_window(ctx):
    """A single inverter input holds every module: its group's window is the
    generator's, and on a one-plane facade (no module occluders either way)
    every output equals the plain evaluation bit for bit."""
    w = mini_facade()
    gid = pv3d.load_workload(ctx, w)
    a = run_gpu(ctx, gid, w)
    b = run_gpu(ctx, gid, w, window_groups=pv3d.PV3D_WINDOWS_PER_ARRAY)
    for k in ("energy", "energy_unshaded", "power", "power_unshaded", "cell_counts", "sample_bits"):
        assert np.array_equal(a[k], b[k]), k
    ctx.release(gid)


def test_window_groups_rejected(ctx):
    w = mini_tracker()
    # modules of tracker 0 split in two runs
    m = w.gen.n_modules
    order = np.r_[0, 24:m, 1:24]
    for f in ("origin", "u", "v", "cells_u", "cells_v", "pitch", "layout", "tracker", "string"):
        setattr(w.gen, f, getattr(w.gen, f)[order])
    gid = pv3d.load_workload(ctx, w)
    with pytest.raises(pv3d.PV3DError):
        ctx.evaluate(gid, n=w.n, map_res=256, window_groups=pv3d.PV3D_WINDOWS_PER_TRACKER)
    with pytest.raises(pv3d.PV3DError):  # string outputs
        ctx.evaluate(gid, n=w.n, map_res=256, window_groups=pv3d.PV3D_WINDOWS_PER_STRING,
                     outputs=("energy", "string_energy"))
    with pytest.raises(pv3d.PV3DError):  # unknown mode
        ctx.evaluate(gid, n=w.n, map_res=256, window_groups=7)
    ctx.release(gid)
