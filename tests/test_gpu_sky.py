"""GPU checks of the inputs made on the device and of the sky map:

* the clear-sky sun table (pv3d_set_sun_clear_sky, FP64 kernels) equals the
  FP64 oracle's table (solar time, Cooper declination, Meinel beam with the
  Kasten-Young air mass) step for step;
* ideal tracker poses made with it give the oracle's unshaded power;
* the effective-shading map over the sky (Fig. 6) equals the oracle's binning
  of the GPU's own per-step powers, and its total loss the oracle's within
  0.1 % absolute."""
import math

import numpy as np
import pytest

import oracle
from paper_1410_5780_gb300 import pv3d, scenes as S

from parity import LOSS_PP, loss_pp, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    pv3d.load(build_if_missing=True)
    c = pv3d.Context(device=0)
    yield c
    c.close()


@pytest.mark.parametrize("lat,step_h,day_first,n_days,daylight", [(40.0, 0.25, 1, 365, True), (-33.5, 1.0, 100, 30, False),
                                                                  (64.0, 0.5, 170, 10, True), (0.0, 1.0 / 3.0, 81, 2, True)])
def test_sun_table_equals_oracle(ctx, lat, step_h, day_first, n_days, daylight):
    w = S.make_tiny()
    gid = pv3d.load_workload(ctx, w)
    n = ctx.set_sun_clear_sky(gid, lat, step_h, day_first=day_first, n_days=n_days, daylight_only=daylight)
    xyz, dni, dhi, dt = ctx.sun_table(gid)
    oxyz, odni, odhi = oracle.sun_table(lat, day_first, n_days, step_h, daylight_only=daylight)
    assert n == oxyz.shape[0]
    np.testing.assert_allclose(xyz, oxyz, rtol=0, atol=1e-12)
    np.testing.assert_allclose(dni, odni, rtol=2e-7, atol=1e-4)
    np.testing.assert_allclose(dhi, odhi, rtol=2e-7, atol=1e-4)
    assert np.all(dt == np.float32(step_h))
    ctx.release(gid)


def test_ideal_tracker_poses_unshaded_power(ctx):
    w = S.make_random_small(41, n_mods=5, n_steps=4, n=2, map_res=512, tracked=True)
    gid = pv3d.load_workload(ctx, w)
    n = ctx.set_sun_clear_sky(gid, 40.0, 1.0, day_first=60, n_days=4, tracker_tilt_max_deg=70.0)
    xyz, dni, dhi, dt = ctx.sun_table(gid)
    g = run_gpu(ctx, gid, w, outputs=("power_unshaded",))
    # the oracle's PV model with zero shading, on the same sun table and the pose rule
    az = np.arctan2(xyz[:, 0], xyz[:, 1])
    tilt = np.minimum(np.arccos(np.clip(xyz[:, 2], -1, 1)), math.radians(70.0))
    poses = np.repeat(np.stack([az, tilt], -1)[:, None, :], w.gen.pivots.shape[0], axis=1).astype(np.float32)
    w2 = S.Workload(w.name, w.scene, w.gen, S.Sun(xyz=xyz, dni=dni, dhi=dhi, dt_h=dt), poses, w.n, w.map_res)
    C = int((w.gen.cells_u * w.gen.cells_v).sum())
    pu = oracle.power_from_counts(w2, np.arange(n), np.arange(w.gen.n_modules), np.zeros((n, C), np.int32))
    assert np.all(np.abs(g["power_unshaded"] - pu) <= 1e-4 * np.maximum(pu, 1.0) + 2e-3), np.abs(g["power_unshaded"] - pu).max()
    ctx.release(gid)


def test_sky_map(ctx):
    w = S.make_facade(seed=17, n=4, map_res=2048, n_buildings=20, n_trees=8, n_poles=4, floors=3, per_floor=8,
                      target_tris=8000, days=np.array([10, 80, 170, 260, 340]), radius=100.0)
    gid = pv3d.load_workload(ctx, w)
    g = ctx.evaluate(gid, n=w.n, map_res=w.map_res, chunk_steps=9, outputs=("power", "power_unshaded"),
                     device=False, heat_bins=(36, 9))
    p = g["power"].astype(np.float64).sum(1); pu = g["power_unshaded"].astype(np.float64).sum(1)
    e, eu, cnt = oracle.heat_map(w.sun.xyz, p, pu, w.sun.dt_h, 36, 9)
    np.testing.assert_array_equal(g["heat_steps"], cnt)
    np.testing.assert_allclose(g["heat_energy"], e, rtol=1e-5, atol=1e-3)
    np.testing.assert_allclose(g["heat_energy_unshaded"], eu, rtol=1e-5, atol=1e-3)
    assert cnt.sum() == int((w.sun.xyz[:, 2] > 0).sum()) and (cnt > 0).sum() > 10
    o = oracle.evaluate_workload(w, want_mask=False)
    oe, oeu, ocnt = oracle.heat_map(w.sun.xyz, o["power"].sum(1), o["power_unshaded"].sum(1), w.sun.dt_h, 36, 9)
    np.testing.assert_array_equal(ocnt, cnt)
    assert abs(loss_pp(g["heat_energy"].sum(), g["heat_energy_unshaded"].sum()) - loss_pp(oe.sum(), oeu.sum())) <= LOSS_PP
    ctx.release(gid)
