"""Served and batched evaluation (continuous batching over shared waves).

Each result must equal, bit for bit, the same evaluation run alone: flags are
per (job, step) and integer, and every job's energy sums run in its own step
order whatever else shares the wave.
"""
import time

import numpy as np
import pytest

from paper_1410_5780_gb300 import pv3d, scenes as S

pytestmark = pytest.mark.gpu

OUTS = ("energy", "energy_unshaded", "power", "power_unshaded", "cell_counts", "sample_bits", "cell_beam_loss")


def _workloads():
    return [
        S.make_tiny(day=355, n=4, map_res=1024),
        S.make_random_small(201, n_mods=6, n_steps=40, n=3, map_res=512),
        S.make_random_small(202, n_mods=5, n_steps=33, n=4, map_res=1024, tracked=True),
        S.make_facade(seed=23, n=4, map_res=1024, n_buildings=10, n_trees=5, n_poles=3, floors=2, per_floor=5,
                      target_tris=3000, days=np.array([30, 120, 250]), radius=70.0),
        S.make_tracker(seed=24, n=2, map_res=1024, grid=(3, 2), terrain_n=48, spacing=1.5, n_pylons=1, step_h=1.0,
                       days=np.array([100, 280])),
    ]


def _np(d):
    out = {}
    for k, v in d.items():
        if hasattr(v, "cpu"):
            a = v.cpu().numpy()
            out[k] = a.view(np.uint64) if k == "sample_bits" else a
        else:
            out[k] = v
    return out


def test_served_mix_equals_alone():
    import torch
    ws = _workloads()
    with pv3d.Context(device=0, chunk_steps=16) as ctx:
        gids = [pv3d.load_workload(ctx, w) for w in ws]
        alone = []
        for w, g in zip(ws, gids):
            alone.append(_np(ctx.evaluate(g, n=w.n, map_res=w.map_res, outputs=OUTS)))
        torch.cuda.synchronize()
        reqs = [ctx.submit(g, n=w.n, map_res=w.map_res, outputs=OUTS) for w, g in zip(ws, gids)]
        for rid, _ in reqs:
            assert ctx.poll(rid, timeout_ms=-1) == pv3d.PV3D_OK
        torch.cuda.synchronize()
        for (rid, arrays), a, w in zip(reqs, alone, ws):
            b = _np(arrays)
            for k in OUTS:
                np.testing.assert_array_equal(a[k], b[k], err_msg=f"{w.name}:{k}")
            assert b["tests"] == a["tests"]
            assert b["latency_ms"] > 0


def test_continuous_batching_short_requests_join_a_running_long_one():
    ws = _workloads()
    long_w = S.make_facade(seed=31, n=4, map_res=2048, n_buildings=30, n_trees=10, n_poles=4, floors=4,
                           per_floor=10, target_tris=12000)
    with pv3d.Context(device=0, chunk_steps=32) as ctx:
        g_long = pv3d.load_workload(ctx, long_w)
        g_short = [pv3d.load_workload(ctx, w) for w in ws[:3]]
        ref = [_np(ctx.evaluate(g, n=w.n, map_res=w.map_res, outputs=OUTS, device=False)) for w, g in
               zip(ws[:3], g_short)]
        rid_long, _ = ctx.submit(g_long, n=long_w.n, map_res=long_w.map_res)
        time.sleep(0.02)
        shorts = [ctx.submit(g, n=w.n, map_res=w.map_res, outputs=OUTS, device=False) for w, g in
                  zip(ws[:3], g_short)]
        done_order = []
        pending = {rid for rid, _ in shorts} | {rid_long}
        t0 = time.time()
        while pending and time.time() - t0 < 120:
            for rid in list(pending):
                rc = ctx.poll(rid, timeout_ms=1)
                if rc == pv3d.PV3D_OK:
                    done_order.append(rid)
                    pending.discard(rid)
                else:
                    assert rc == pv3d.PV3D_E_PENDING
        assert not pending
        # the short requests were admitted while the long one ran and finished first
        assert done_order[-1] == rid_long
        for (rid, arrays), a in zip(shorts, ref):
            for k in OUTS:
                np.testing.assert_array_equal(a[k], arrays[k], err_msg=k)


def test_admission_rejects_requests_over_the_budget():
    w = S.make_tiny(day=355)
    with pv3d.Context(device=0, hbm_budget_bytes=4096) as ctx:
        gid = pv3d.load_workload(ctx, w)
        with pytest.raises(pv3d.PV3DError) as e:
            ctx.submit(gid, n=4)
        assert e.value.code == pv3d.PV3D_E_ADMISSION


def test_poll_wait_is_bounded_and_release_refuses_ids_in_use():
    w = S.make_facade(seed=41, n=8, map_res=4096, n_buildings=20, n_trees=6, n_poles=4, floors=4, per_floor=10,
                      target_tris=10000)
    with pv3d.Context(device=0) as ctx:
        gid = pv3d.load_workload(ctx, w)
        rid, _ = ctx.submit(gid, n=w.n, map_res=w.map_res)
        t0 = time.time()
        rc = ctx.poll(rid, timeout_ms=1)
        assert time.time() - t0 < 5.0
        if rc == pv3d.PV3D_E_PENDING:
            with pytest.raises(pv3d.PV3DError):
                ctx.release(gid)
        assert ctx.poll(rid, timeout_ms=-1) in (pv3d.PV3D_OK, rc)
        ctx.release(gid)


def test_evaluate_batch_equals_alone():
    ws = _workloads()[:3]
    with pv3d.Context(device=0, chunk_steps=8) as ctx:
        gids = [pv3d.load_workload(ctx, w) for w in ws]
        alone = [_np(ctx.evaluate(g, n=4, map_res=1024, outputs=("energy", "energy_unshaded", "cell_counts")))
                 for g in gids]
        batch = ctx.evaluate_batch(gids, n=4, map_res=1024, outputs=("energy", "energy_unshaded", "cell_counts"))
        for a, b in zip(alone, batch):
            b = _np(b)
            for k in ("energy", "energy_unshaded", "cell_counts"):
                np.testing.assert_array_equal(a[k], b[k])


def test_served_strings_arrays_and_diffuse_equal_alone():
    """Served requests with series-string and parallel-array outputs and the
    diffuse term shaded, mixed with a plain request, equal the same
    evaluations run alone bit for bit (their string and array Kahan sums run
    in step order in the request's own accumulators), with device and with
    host outputs."""
    import torch
    w = S.make_facade(seed=25, n=3, map_res=1024, n_buildings=10, n_trees=5, n_poles=3, floors=2, per_floor=6,
                      target_tris=3000, days=np.array([30, 120, 250]), radius=70.0)
    w.gen.string = (np.arange(w.gen.n_modules) // 3).astype(np.int32)
    w.gen.array = (np.arange(w.gen.n_modules) // 6).astype(np.int32)
    other = S.make_random_small(203, n_mods=5, n_steps=30, n=3, map_res=512)
    outs = ("energy", "energy_unshaded", "power", "string_energy", "string_energy_unshaded", "string_power",
            "array_energy", "array_energy_unshaded", "array_power")
    with pv3d.Context(device=0, chunk_steps=16) as ctx:
        gid = pv3d.load_workload(ctx, w)
        ctx.sky_view(gid, rings=4, sectors=12, n=2, map_res=512)
        g2 = pv3d.load_workload(ctx, other)
        for device in (True, False):
            alone = _np(ctx.evaluate(gid, n=w.n, map_res=w.map_res, outputs=outs, device=device,
                                     diffuse_shading=True))
            torch.cuda.synchronize()
            r_other = ctx.submit(g2, n=other.n, map_res=other.map_res)
            rid, arrays = ctx.submit(gid, n=w.n, map_res=w.map_res, outputs=outs, device=device,
                                     diffuse_shading=True)
            assert ctx.poll(r_other[0], timeout_ms=-1) == pv3d.PV3D_OK
            assert ctx.poll(rid, timeout_ms=-1) == pv3d.PV3D_OK
            torch.cuda.synchronize()
            b = _np(arrays)
            assert b["string_energy"].shape == (len(ctx.string_ids(gid)),)
            assert b["array_energy"].shape == (len(ctx.array_ids(gid)),)
            for k in outs:
                np.testing.assert_array_equal(alone[k], b[k], err_msg=f"device={device}:{k}")
            assert b["string_energy"].sum() > 0 and b["array_energy"].sum() > 0
