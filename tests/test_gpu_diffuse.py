"""GPU parity of diffuse shading (pv3d_sky_view): per-cell shares of the
cosine-weighted sky hidden by the scene, from depth tests toward the sky
patches, against the FP64 oracle's ray tests toward the same patches; a long
wall against its closed-form view factor; tracked modules per pose bin; and
the PV model with the diffuse term shaded, on the GPU's own counts and
fractions."""
import math

import numpy as np
import pytest

import oracle
from paper_1410_5780_gb300 import pv3d, scenes as S

from parity import run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    pv3d.load(build_if_missing=True)
    c = pv3d.Context(device=0)
    yield c
    c.close()


def oracle_fractions(w, rings, sectors, n, map_res):
    xyz, _ = oracle.sky_patches(rings, sectors)
    sun = S.Sun(xyz=xyz, dni=np.ones(len(xyz), np.float32), dhi=np.zeros(len(xyz), np.float32),
                dt_h=np.ones(len(xyz), np.float32))
    o = oracle.evaluate(w.scene, w.gen, sun, None, n, map_res)
    starts = np.concatenate([[0], np.cumsum(w.gen.cells_u * w.gen.cells_v)])
    normals = np.concatenate([np.repeat(np.cross(w.gen.u[m], w.gen.v[m])[None, :].astype(np.float64),
                                        starts[m + 1] - starts[m], 0) for m in range(w.gen.n_modules)])
    normals /= np.linalg.norm(normals, axis=1, keepdims=True)
    wn = S.Workload(w.name, w.scene, w.gen, sun, None, n, map_res)
    f = oracle.diffuse_shade_fractions(wn, rings, sectors, o["counts"], normals)
    # the bound: masked samples toward each patch, weighted like the fraction
    pxyz, dom = oracle.sky_patches(rings, sectors)
    wgt = dom[:, None] * np.maximum(0.0, pxyz @ normals.T)
    masked = oracle.popcount64(o["mbits"]) / float(n * n)
    bound = (wgt * masked).sum(0) / np.maximum(wgt.sum(0), 1e-300)
    return f, bound


@pytest.mark.parametrize("h,d", [(3.0, 3.0), (10.0, 4.0)])
def test_long_wall(ctx, h, d):
    mb = S.MeshBuilder()
    mb.grid_quad((-200.0, d, 0.0), (400.0, 0.0, 0.0), (0.0, 0.0, h), 40, 1)
    lay = S.Layout(2, 2, 1, np.zeros(4, np.int32))
    gen = S._gen_from_lists([(-0.156, -0.156, 0.0)], [(1.0, 0.0, 0.0)], [(0.0, 1.0, 0.0)], 2, 2, [0], [-1], [0],
                            [lay], np.zeros((0, 3)))
    sun = S.Sun(xyz=np.array([[0.0, 0.0, 1.0]]), dni=np.ones(1, np.float32), dhi=np.ones(1, np.float32),
                dt_h=np.ones(1, np.float32))
    w = S.Workload("wall", mb.build(), gen, sun, None, 4, 1024)
    gid = pv3d.load_workload(ctx, w)
    f = ctx.sky_view(gid, rings=18, sectors=72, n=4, map_res=1024)
    expect = 0.5 * (1 - d / math.hypot(d, h))
    assert np.all(np.abs(f - expect) < 0.015), (f, expect)
    fo, bound = oracle_fractions(w, 18, 72, 4, 1024)
    assert np.all(np.abs(f - fo) <= bound + 0.005), (f, fo, bound)
    ctx.release(gid)


def test_facade_fractions_and_pv_model(ctx):
    w = S.make_facade(seed=23, n=3, map_res=1024, n_buildings=12, n_trees=6, n_poles=4, floors=2, per_floor=6,
                      target_tris=4000, days=np.array([20, 110, 200, 300]), radius=60.0)
    gid = pv3d.load_workload(ctx, w)
    f = ctx.sky_view(gid, rings=9, sectors=36, n=3, map_res=1024)
    fo, bound = oracle_fractions(w, 9, 36, 3, 1024)
    assert np.all(np.abs(f - fo) <= bound + 0.01), np.abs(f - fo).max()
    assert f.max() > 0.05  # the buildings and trees hide part of the sky
    # PV model with the diffuse term shaded, on the GPU's counts and fractions
    g = ctx.evaluate(gid, n=w.n, map_res=w.map_res, outputs=("cell_counts", "power", "energy", "energy_unshaded"),
                     device=False, diffuse_shading=True)
    g0 = ctx.evaluate(gid, n=w.n, map_res=w.map_res, outputs=("energy",), device=False)
    assert np.all(g["energy"] <= g0["energy"] + 1e-6) and g["energy"].sum() < g0["energy"].sum()
    starts = np.concatenate([[0], np.cumsum(w.gen.cells_u * w.gen.cells_v)])
    lay = w.gen.layouts[0]
    rng = np.random.default_rng(1)
    for st in rng.choice(np.flatnonzero(w.sun.xyz[:, 2] > 0), 12, replace=False):
        s = w.sun.xyz[st]
        for m in range(w.gen.n_modules):
            nrm = np.cross(w.gen.u[m], w.gen.v[m]).astype(np.float64)
            nrm /= np.linalg.norm(nrm)
            beam = float(w.sun.dni[st]) * max(0.0, float(nrm @ s))
            diff = float(w.sun.dhi[st]) * (1 + nrm[2]) / 2
            c0, c1 = starts[m], starts[m + 1]
            fc = g["cell_counts"][st, c0:c1] / float(w.n * w.n)
            G = beam * (1 - fc) + diff * (1 - f[c0:c1].astype(np.float64))
            p = oracle.module_pmpp(G, lay.cell_sub, lay.n_sub)
            assert abs(g["power"][st, m] - p) <= 1e-4 * max(p, 1.0) + 1e-3, (st, m, g["power"][st, m], p)
    with pytest.raises(pv3d.PV3DError):
        ctx.evaluate(987654, n=2, diffuse_shading=True)
    ctx.release(gid)


def test_tracked_fractions_per_pose_bin_and_pv_model(ctx):
    """Tracked modules: fractions per pose bin (a step's bin is the first
    tracker's pose; every tracker at the bin's centre pose for the sky view)
    against the oracle's exact rays toward the same patches at the same
    poses, and the PV model with the diffuse term shaded by the row of each
    step's bin and the module's own tilt at the step."""
    w = S.make_tracker(seed=29, n=3, map_res=512, grid=(3, 2), terrain_n=48, spacing=1.5, relief=2.0, n_pylons=1,
                       step_h=2.0, days=np.array([40, 200]))
    gid = pv3d.load_workload(ctx, w)
    rings, sectors, n_az, n_tilt = 4, 12, 4, 2
    f = ctx.sky_view(gid, rings=rings, sectors=sectors, n=3, map_res=512, pose_az_bins=n_az, pose_tilt_bins=n_tilt)
    assert f.shape == (n_az * n_tilt, w.gen.n_cells)
    fo, masked, step_bin = oracle.tracked_diffuse_fractions(w, rings, sectors, n_az, n_tilt, 3, 512)
    assert len(fo) >= 2
    for b in range(n_az * n_tilt):
        if b in fo:
            assert np.all(np.abs(f[b] - fo[b]) <= masked[b] + 0.01), (b, np.abs(f[b] - fo[b]).max())
        else:
            assert not f[b].any()
    assert max(float(fo[b].max()) for b in fo) > 0.02  # neighbouring tables and the ground hide some sky
    g = ctx.evaluate(gid, n=w.n, map_res=w.map_res, outputs=("cell_counts", "power", "energy"), device=False,
                     diffuse_shading=True)
    g0 = ctx.evaluate(gid, n=w.n, map_res=w.map_res, outputs=("energy",), device=False)
    assert g["energy"].sum() < g0["energy"].sum()
    starts = np.concatenate([[0], np.cumsum(w.gen.cells_u * w.gen.cells_v)])
    lay = w.gen.layouts[0]
    rng = np.random.default_rng(2)
    lit = np.flatnonzero(w.sun.xyz[:, 2] > 0)
    for st in rng.choice(lit, min(8, len(lit)), replace=False):
        s = w.sun.xyz[st]
        for m in rng.choice(w.gen.n_modules, 12, replace=False):
            nrm = oracle.module_normal(w.gen, w.poses, int(st), int(m))
            beam = float(w.sun.dni[st]) * max(0.0, float(nrm @ s))
            diff = float(w.sun.dhi[st]) * (1 + nrm[2]) / 2
            c0, c1 = starts[m], starts[m + 1]
            fc = g["cell_counts"][st, c0:c1] / float(w.n * w.n)
            G = beam * (1 - fc) + diff * (1 - f[step_bin[st], c0:c1].astype(np.float64))
            p = oracle.module_pmpp(G, lay.cell_sub, lay.n_sub)
            assert abs(g["power"][st, m] - p) <= 1e-4 * max(p, 1.0) + 1e-3, (st, m, g["power"][st, m], p)
    # a new pose table drops the fractions
    ctx.set_poses(gid, w.poses)
    with pytest.raises(pv3d.PV3DError):
        ctx.evaluate(gid, n=2, diffuse_shading=True)
    ctx.release(gid)
