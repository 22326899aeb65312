"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Small workloads (tiny two-module case, random scenes, reduced facade and
tracker plants) are compared in full; the full-size facade (R = 4096, 8x8
samples) and tracker plant (R = 8192, 4x4 samples) are compared on sampled
sun steps and modules in the launch configuration the benchmark uses.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1410_5780_gb300 import pv3d, scenes as S

from parity import FLAG_AGREEMENT, LOSS_PP, compare, energy_checks, loss_pp, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    pv3d.load(build_if_missing=True)
    c = pv3d.Context(device=0)
    yield c
    c.close()


def full_check(ctx, w, chunk_steps=0, strict_loss=True):
    """Flags, cell fractions and energies over every step of ``w``.  With
    ``strict_loss`` the total and per-module loss must match the oracle's
    within 0.1 % absolute; otherwise (coarse maps, few random steps) the loss
    must lie in the oracle's masked-sample envelope."""
    gid = pv3d.load_workload(ctx, w)
    g = run_gpu(ctx, gid, w, chunk_steps=chunk_steps)
    o = oracle.evaluate_workload(w)
    st = compare(w, g, o, np.arange(w.sun.n_steps))
    assert st["agree"] >= FLAG_AGREEMENT, st
    assert st["cell_ok"] == 1.0, st
    energy_checks(w, g, o, np.arange(w.sun.n_steps))
    if strict_loss:
        lg, lo = loss_pp(g["energy"], g["energy_unshaded"]), loss_pp(o["energy"], o["energy_unshaded"])
        assert abs(lg - lo) <= LOSS_PP, (lg, lo)
        for m in range(w.gen.n_modules):
            assert abs(loss_pp(g["energy"][m], g["energy_unshaded"][m])
                       - loss_pp(o["energy"][m], o["energy_unshaded"][m])) <= LOSS_PP
    assert g["tests"] == int((w.sun.xyz[:, 2] > 0).sum()) * w.samples_per_step
    ctx.release(gid)
    return g, o, st


@pytest.mark.parametrize("day", [172, 355, 80])
def test_tiny_full(ctx, day):
    w = S.make_tiny(day=day)
    g, o, st = full_check(ctx, w)
    if day == 355:
        assert o["counts"].sum() > 1000  # the box shades the modules in winter


@pytest.mark.parametrize("seed,tracked", [(101, False), (102, True), (103, False), (104, True), (105, False)])
def test_random_small(ctx, seed, tracked):
    w = S.make_random_small(seed, n_mods=6, n_steps=12, n=3, map_res=512, tracked=tracked)
    full_check(ctx, w, chunk_steps=5, strict_loss=False)


def test_many_substring_modules(ctx):
    """Modules of 12 bypass substrings (two per cell column) among 3-substring
    modules: the PV kernel evaluates up to 8 substrings per lane and falls back
    to one module per warp otherwise; with 70 modules a step, its 32-item
    batches take both forms, and batches cross steps."""
    w = S.make_random_small(106, n_mods=70, n_steps=6, n=3, map_res=512)
    g = w.gen
    cu, cv = g.layouts[0].cells_u, g.layouts[0].cells_v
    col = np.tile(np.arange(cu), cv)
    half = (np.repeat(np.arange(cv), cu) >= cv // 2).astype(np.int32)
    g.layouts.append(S.Layout(cu, cv, 2 * cu, (2 * col + half).astype(np.int32)))
    g.layout[:2] = 1
    full_check(ctx, w, chunk_steps=4, strict_loss=False)


def test_mini_facade(ctx):
    w = S.make_facade(seed=7, n=4, map_res=1024, n_buildings=12, n_trees=6, n_poles=4, floors=2, per_floor=6,
                      target_tris=4000, days=np.array([20, 110, 200, 300]), radius=80.0)
    full_check(ctx, w)


def test_mini_tracker(ctx):
    w = S.make_tracker(seed=9, n=4, map_res=1024, grid=(4, 3), terrain_n=64, spacing=1.5, n_pylons=2,
                       step_h=1.0, days=np.array([30, 172, 300]))
    full_check(ctx, w, strict_loss=False)


@pytest.mark.parametrize("make", ["tiny_dec21", "mini_tracker"])
def test_cell_beam_loss_vs_oracle(ctx, make):
    """Per-cell annual beam irradiation lost to shading (Section 2 step 4).
    1. The GPU's Kahan FP32 sums equal the FP64 sum over steps of
       DNI cos dt f_c on the GPU's own cell counts.
    2. Every cell whose unmasked flags agree with the oracle's at every step
       lies between the oracle's sums with its masked samples forced lit and
       forced shaded."""
    if make == "tiny_dec21":
        w = S.make_tiny(day=355)
    else:
        w = S.make_tracker(seed=9, n=4, map_res=1024, grid=(4, 3), terrain_n=64, spacing=1.5, n_pylons=2,
                           step_h=1.0, days=np.array([30, 172, 300]))
    gid = pv3d.load_workload(ctx, w)
    g = run_gpu(ctx, gid, w, outputs=("cell_beam_loss", "cell_counts", "sample_bits"))
    ctx.release(gid)
    o = oracle.evaluate_workload(w)
    steps, mods = o["steps"], o["modules"]
    gl = g["cell_beam_loss"].astype(np.float64)
    own = oracle.cell_beam_loss_from_counts(w, steps, mods, g["cell_counts"].astype(np.int64), o["cos_inc"])
    assert own.max() > 0
    tol = 1e-4 * np.maximum(np.abs(own), 1.0)
    assert np.all(np.abs(gl - own) <= tol), np.abs(gl - own).max()
    ob, mb, gb = o["bits"], o["mbits"], g["sample_bits"]
    lo = oracle.cell_beam_loss_from_counts(w, steps, mods, oracle.popcount64(ob & ~mb), o["cos_inc"])
    hi = oracle.cell_beam_loss_from_counts(w, steps, mods, oracle.popcount64(ob | mb), o["cos_inc"])
    agree = (((gb ^ ob) & ~mb) == 0).all(0)
    assert agree.mean() >= 0.99, agree.mean()
    tol = 1e-4 * np.maximum(hi, 1.0)
    ok = (gl >= lo - tol) & (gl <= hi + tol)
    assert ok[agree].all(), (np.flatnonzero(~ok & agree)[:5], gl[~ok & agree][:5], lo[~ok & agree][:5])
    # the cells the oracle shades with no ambiguity carry beam loss on the GPU too
    assert (gl[agree & (lo > 0)] > 0).all()


@pytest.mark.parametrize("tile,fmt,path", [(32, 0, 0), (64, 1, 0), (32, 1, 1), (64, 0, 1), (128, 0, 0), (128, 1, 1)])
def test_tile_depth_format_and_path(tile, fmt, path):
    w = S.make_random_small(111, n_mods=6, n_steps=10, n=4, map_res=1024, tracked=True)
    o = oracle.evaluate_workload(w)
    with pv3d.Context(device=0, tile=tile, depth_format=fmt) as c2:
        gid = pv3d.load_workload(c2, w)
        g = run_gpu(c2, gid, w, path=path)
        st = compare(w, g, o, np.arange(w.sun.n_steps))
        assert st["agree"] >= FLAG_AGREEMENT, (tile, fmt, path, st)
        energy_checks(w, g, o, np.arange(w.sun.n_steps))


@pytest.mark.parametrize("make", ["tracker_mini", "facade_mini", "random"])
def test_fused_and_map_paths_bit_identical(ctx, make):
    """The fused path (tests inside the raster CTA) and the map path (HBM map +
    gather kernel) read the same texels with the same arithmetic."""
    if make == "tracker_mini":
        w = S.make_tracker(seed=19, n=4, map_res=2048, grid=(5, 4), terrain_n=96, spacing=1.5, n_pylons=3,
                           step_h=0.5, days=np.array([15, 100, 200]))
    elif make == "facade_mini":
        w = S.make_facade(seed=17, n=8, map_res=2048, n_buildings=20, n_trees=8, n_poles=4, floors=3,
                          per_floor=8, target_tris=8000, days=np.array([10, 80, 170, 260, 340]), radius=100.0)
    else:
        w = S.make_random_small(23, n_mods=8, n_steps=20, n=5, map_res=512, tracked=True)
    gid = pv3d.load_workload(ctx, w)
    a = run_gpu(ctx, gid, w, path=pv3d.PV3D_PATH_FUSED, chunk_steps=7)
    b = run_gpu(ctx, gid, w, path=pv3d.PV3D_PATH_MAP, chunk_steps=7)
    for k in ("sample_bits", "cell_counts", "power", "power_unshaded", "energy", "energy_unshaded"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert a["cell_counts"].sum() > 0
    ctx.release(gid)


def _sampled_full_size(ctx, w, windows, n_mods, seed, chunk_steps=0):
    gid = pv3d.load_workload(ctx, w)
    rng = np.random.default_rng(seed)
    mods = np.sort(rng.choice(w.gen.n_modules, n_mods, replace=False))
    osc = oracle.OracleScene(w.scene.verts, w.scene.tris)
    stats = []
    for b, k in windows:
        g = run_gpu(ctx, gid, w, step_begin=b, step_end=b + k, chunk_steps=chunk_steps,
                    outputs=("sample_bits", "cell_counts", "power", "power_unshaded"))
        o = oracle.evaluate_workload(w, steps=np.arange(b, b + k), modules=mods, oscene=osc)
        st = compare(w, g, o, np.arange(k))
        stats.append(st)
        assert st["agree"] >= FLAG_AGREEMENT, (b, st)
        assert st["cell_ok"] >= 0.999, (b, st)
        energy_checks(w, g, o, np.arange(k))
    ctx.release(gid)
    return stats


def test_facade_full_size_sampled(ctx):
    w = S.make_facade()
    n = w.sun.n_steps
    windows = [(int(0.03 * n), 12), (int(0.48 * n), 12), (int(0.9 * n), 12)]
    stats = _sampled_full_size(ctx, w, windows, n_mods=12, seed=3)
    assert sum(s["n_unmasked"] for s in stats) > 100000


def test_tracker_full_size_sampled(ctx):
    w = S.make_tracker()
    n = w.sun.n_steps
    # early-morning steps (ridge and long inter-tracker shadows) and midday
    windows = [(int(0.2 * n), 6), (int(0.2 * n) + 30, 4), (int(0.7 * n) + 11, 4)]
    stats = _sampled_full_size(ctx, w, windows, n_mods=24, seed=4)
    assert sum(s["n_unmasked"] for s in stats) > 50000


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_empty_scene_zero_loss(ctx):
    w = S.make_tiny(day=355)
    w.scene = S.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32))
    gid = pv3d.load_workload(ctx, w)
    g = run_gpu(ctx, gid, w)
    assert g["cell_counts"].sum() == 0
    np.testing.assert_array_equal(g["power"], g["power_unshaded"])
    ctx.release(gid)


def test_night_steps_skipped_and_ragged_chunks(ctx):
    w = S.make_random_small(121, n_mods=4, n_steps=9, n=2, map_res=256)
    # interleave night steps
    night = np.array([[0.3, 0.1, -0.2]])
    night /= np.linalg.norm(night)
    xyz = np.concatenate([w.sun.xyz[:4], night, w.sun.xyz[4:], night])
    w.sun = S.Sun(xyz=xyz, dni=np.concatenate([w.sun.dni[:4], [0], w.sun.dni[4:], [0]]).astype(np.float32),
                  dhi=np.concatenate([w.sun.dhi[:4], [0], w.sun.dhi[4:], [0]]).astype(np.float32),
                  dt_h=np.ones(len(xyz), np.float32))
    for k in (1, 3, 4, 16):
        gid = pv3d.load_workload(ctx, w)
        g = run_gpu(ctx, gid, w, chunk_steps=k)
        assert g["tests"] == 9 * w.samples_per_step
        assert g["steps_lit"] == 9
        assert g["power"][4].sum() == 0 and g["power"][-1].sum() == 0
        o = oracle.evaluate_workload(w)
        st = compare(w, g, o, np.arange(w.sun.n_steps))
        assert st["agree"] >= FLAG_AGREEMENT
        ctx.release(gid)


@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_samples_per_side(ctx, n):
    w = S.make_tiny(day=355, n=n)
    full_check(ctx, w, chunk_steps=7)


def test_single_module_grazing_sun(ctx):
    w = S.make_tiny(day=355)
    # a dawn sun below 2 degrees of elevation uses the FP64 light frame
    el = [0.5, 1.5, 1.99, 2.5, 10.0]
    az = math.radians(125.0)
    xyz = np.array([[math.sin(az) * math.cos(math.radians(e)), math.cos(az) * math.cos(math.radians(e)),
                     math.sin(math.radians(e))] for e in el])
    w.sun = S.Sun(xyz=xyz, dni=np.full(len(el), 300, np.float32), dhi=np.full(len(el), 30, np.float32),
                  dt_h=np.ones(len(el), np.float32))
    full_check(ctx, w)


def test_kahan_energy_vs_fp64_sum(ctx):
    w = S.make_facade(seed=5, n=2, map_res=512, n_buildings=6, n_trees=3, n_poles=2, floors=1, per_floor=4,
                      target_tris=1500, radius=60.0)
    gid = pv3d.load_workload(ctx, w)
    g = run_gpu(ctx, gid, w, outputs=("energy", "energy_unshaded", "power", "power_unshaded"))
    dt = w.sun.dt_h.astype(np.float64)
    e64 = (g["power"].astype(np.float64) * dt[:, None]).sum(0)
    rel = np.abs(g["energy"] - e64) / np.maximum(e64, 1e-9)
    assert rel.max() <= 1e-6, rel.max()
    ctx.release(gid)


def test_determinism_and_host_outputs(ctx):
    w = S.make_random_small(131, n_mods=6, n_steps=10, n=3, map_res=512, tracked=True)
    gid = pv3d.load_workload(ctx, w)
    a = run_gpu(ctx, gid, w)
    b = run_gpu(ctx, gid, w)
    h = run_gpu(ctx, gid, w, device=False)
    for k in ("energy", "energy_unshaded", "power", "sample_bits", "cell_counts"):
        np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(a[k], h[k])
    ctx.release(gid)


def test_facade_year_subsample_loss(ctx):
    """Full-size facade (R = 4096, 8x8 samples, all 200 modules) on every 8th
    day of the year: the loss over those days within 0.1 % of the oracle's."""
    w = S.make_facade(days=np.arange(4, 366, 8))
    gid = pv3d.load_workload(ctx, w)
    g = run_gpu(ctx, gid, w, outputs=("energy", "energy_unshaded"))
    o = oracle.evaluate_workload(w, want_mask=False)
    lg, lo = loss_pp(g["energy"], g["energy_unshaded"]), loss_pp(o["energy"], o["energy_unshaded"])
    assert abs(lg - lo) <= LOSS_PP, (lg, lo)
    ctx.release(gid)


def test_tracker_year_subsample_loss(ctx):
    """Full-size tracker plant (R = 8192, 4x4 samples) on every 16th day: the
    loss of 300 sampled modules within 0.1 % of the oracle's."""
    w = S.make_tracker(days=np.arange(3, 366, 16))
    gid = pv3d.load_workload(ctx, w)
    g = run_gpu(ctx, gid, w, outputs=("power", "power_unshaded"))
    mods = np.sort(np.random.default_rng(8).choice(w.gen.n_modules, 300, replace=False))
    o = oracle.evaluate_workload(w, modules=mods, want_mask=False)
    dt = w.sun.dt_h.astype(np.float64)[:, None]
    lg = loss_pp((g["power"][:, mods] * dt).sum(), (g["power_unshaded"][:, mods] * dt).sum())
    lo = loss_pp(o["energy"], o["energy_unshaded"])
    assert abs(lg - lo) <= LOSS_PP, (lg, lo)
    ctx.release(gid)


def test_invalid_inputs_rejected(ctx):
    w = S.make_tiny()
    bad = w.scene.verts.copy()
    bad[0, 0] = np.nan
    with pytest.raises(pv3d.PV3DError) as e:
        ctx.scene_load(bad, w.scene.tris)
    assert e.value.code == pv3d.PV3D_E_INVALID
    with pytest.raises(pv3d.PV3DError):
        ctx.scene_load(w.scene.verts, w.scene.tris + 100)
    sid = ctx.scene_load(w.scene.verts, w.scene.tris)
    gid = ctx.generator_define(sid, w.gen)
    with pytest.raises(pv3d.PV3DError):
        ctx.set_sun(gid, w.sun.xyz * 1.01, w.sun.dni, w.sun.dhi, w.sun.dt_h)
    with pytest.raises(pv3d.PV3DError):  # no sun table yet
        ctx.evaluate(gid, n=2)
    ctx.set_sun(gid, w.sun.xyz, w.sun.dni, w.sun.dhi, w.sun.dt_h)
    with pytest.raises(pv3d.PV3DError):
        ctx.evaluate(gid, n=16)
    with pytest.raises(pv3d.PV3DError):
        ctx.evaluate(gid, n=9, outputs=("sample_bits",))
    with pytest.raises(pv3d.PV3DError):
        ctx.evaluate(gid, n=2, map_res=1000)
    bad_gen = S.make_tiny().gen
    bad_gen.layouts = [S.Layout(6, 10, 3, np.zeros(60, np.int32))]  # substrings 1, 2 own no cell
    with pytest.raises(pv3d.PV3DError):
        ctx.generator_define(sid, bad_gen)
    with pytest.raises(pv3d.PV3DError) as e:
        ctx.evaluate(987654, n=2)
    assert e.value.code == pv3d.PV3D_E_NOTFOUND
    ctx.release(sid)


def test_stepped_tracker_table_shades_itself(ctx):
    """Modules of one tracker table that do not share a plane (a row raised
    0.3 m along the table's normal, overlapping the row below like shingles)
    shade one another; modules that share one plane cannot, and the binning
    leaves their triangles out of the tiles whose receivers all lie in that
    plane.  Both against the FP64 oracle at non-normal incidence (tilt limit
    30 deg, low suns)."""
    cu, cv = 6, 10
    p = S.CELL_PITCH
    w0, h0 = cu * p, cv * p
    origins = [(-w0 - 0.01, -h0, 0.0), (0.01, -h0, 0.0),                 # lower row, coplanar pair
               (-w0 - 0.01, -0.25, 0.3), (0.01, -0.25, 0.3)]             # raised row, overlapping by 0.25 m
    lay = S.standard_layout(cu, cv, 3)
    gen = S._gen_from_lists(origins, [(1.0, 0.0, 0.0)] * 4, [(0.0, 1.0, 0.0)] * 4, cu, cv, [0] * 4, [0] * 4,
                            list(range(4)), [lay], np.array([[0.0, 0.0, 3.0]]))
    mb = S.MeshBuilder()
    mb.box((6.0, 6.0, 0.0), (6.5, 6.5, 0.5))
    scene = mb.build()
    days, hours = np.array([80, 80, 80, 172, 172, 355, 355, 355]), np.array([8.0, 9.5, 15.0, 7.0, 18.0, 9.0, 12.0, 14.5])
    xyz = S.sun_vectors(40.0, days, hours)
    dni = S.clear_sky_dni(xyz[:, 2]).astype(np.float32)
    sun = S.Sun(xyz=xyz, dni=dni, dhi=(0.1 * dni).astype(np.float32), dt_h=np.ones(len(xyz), np.float32))
    poses = S.ideal_poses(sun, 1, 30.0)
    w = S.Workload("stepped", scene, gen, sun, poses, 4, 1024)
    g, o, st = full_check(ctx, w, strict_loss=False)
    cells = cu * cv
    assert o["counts"][:, :2 * cells].sum() > 100       # the raised row shades the lower one
    assert g["cell_counts"][:, :2 * cells].sum() > 100


@pytest.mark.parametrize("make", ["random", "mini_tracker"])
def test_bin_pool_overflow_regrows(make):
    """A context whose (triangle, tile) pool holds 16 entries overflows on its
    first wave; the kernels stop appending at the pool's end and flag it, and
    the host grows the pool from the demand they counted and reruns.  The
    results must equal those of a context with the default pool bit for bit,
    and meet the oracle criteria."""
    if make == "random":
        w = S.make_random_small(141, n_mods=6, n_steps=10, n=3, map_res=512, tracked=True)
    else:
        w = S.make_tracker(seed=9, n=4, map_res=1024, grid=(4, 3), terrain_n=64, spacing=1.5, n_pylons=2,
                           step_h=1.0, days=np.array([30, 172, 300]))
    with pv3d.Context(device=0, bin_capacity=16) as small, pv3d.Context(device=0) as big:
        a = run_gpu(small, pv3d.load_workload(small, w), w)
        b = run_gpu(big, pv3d.load_workload(big, w), w)
    assert b["binned_tris"] > 16 * b["waves"]  # every wave needs more than the small pool
    for k in ("sample_bits", "cell_counts", "power", "power_unshaded", "energy", "energy_unshaded"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    o = oracle.evaluate_workload(w)
    st = compare(w, a, o, np.arange(w.sun.n_steps))
    assert st["agree"] >= FLAG_AGREEMENT, st
    energy_checks(w, a, o, np.arange(w.sun.n_steps))


def test_maximum_sizes(ctx):
    """The largest sizes the boundary takes: 15 x 15 samples per cell (a cell's
    count reaches 225, the most its one-byte tally holds), a module of 32 x 32
    = 1024 cells (the per-module maximum) with 64 bypass substrings (the
    maximum: each cell column split in two halves), and the largest light window side,
    16384 -- against the oracle's counts cell by cell, and fully shaded cells
    reaching 225."""
    n, cu, cv = 15, 32, 32
    p = 0.05
    mb = S.MeshBuilder()
    mb.box((-0.4, -0.4, 0.0), (1.2, 0.2, 2.0))   # a block over part of the module
    scene = mb.build()
    # substring 2 c + h: cell column c, lower (h = 0) or upper (h = 1) half
    lay = S.Layout(cu, cv, 64, (2 * np.tile(np.arange(cu), cv) + (np.repeat(np.arange(cv), cu) >= cv // 2))
                   .astype(np.int32))
    gen = S._gen_from_lists([(0.0, 0.0, 0.05)], [(1.0, 0.0, 0.0)], [(0.0, 1.0, 0.0)], cu, cv, [0], [-1], [0], [lay],
                            np.zeros((0, 3)))
    gen.pitch = np.full(1, p, np.float32)
    xyz = S.sun_vectors(40.0, np.array([172, 172, 355]), np.array([10.0, 14.0, 12.0]))
    dni = S.clear_sky_dni(xyz[:, 2]).astype(np.float32)
    sun = S.Sun(xyz=xyz, dni=dni, dhi=(0.1 * dni).astype(np.float32), dt_h=np.ones(3, np.float32))
    w = S.Workload("max", scene, gen, sun, None, n, 16384)
    gid = pv3d.load_workload(ctx, w)
    g = run_gpu(ctx, gid, w, outputs=("cell_counts", "power", "energy", "energy_unshaded"))
    ctx.release(gid)
    o = oracle.evaluate_workload(w)
    gc = g["cell_counts"].astype(np.int64)
    oc = o["counts"].astype(np.int64)
    assert oc.max() == n * n and gc.max() == n * n   # fully shaded cells hold 225
    # a texel of 1.6 m / 16382 = 0.1 mm: counts agree except within a few
    # samples of the block's shadow edge
    diff = np.abs(gc - oc)
    assert (diff == 0).mean() >= 0.99, (diff > 0).mean()
    assert diff.max() <= n, diff.max()
    assert oc.sum() > 0 and abs(int(gc.sum()) - int(oc.sum())) <= 0.001 * oc.sum() + n
    # the PV model over 64 substrings on the GPU's own counts
    pc = oracle.power_from_counts(w, np.arange(3), [0], gc.astype(np.int32))
    assert np.all(np.abs(g["power"].astype(np.float64) - pc) <= 1e-4 * np.maximum(pc, 1.0) + 1e-3), (g["power"], pc)
