"""GPU parity of the series-string electrical model (Section 2: modules wired
in series strings, Fig. 2): per step, the string's maximum power from the
GPU's own cell counts equals the FP64 oracle's string model on those counts;
string energies are the Kahan sums of the string powers; the string loss lies
in the oracle's masked-sample envelope; one module per string reproduces the
module outputs."""
import numpy as np
import pytest

import oracle
from paper_1410_5780_gb300 import pv3d, scenes as S

from parity import LOSS_PP, run_gpu

pytestmark = pytest.mark.gpu

OUTS = ("cell_counts", "power", "power_unshaded", "string_power", "string_power_unshaded", "string_energy",
        "string_energy_unshaded", "energy")


@pytest.fixture(scope="module")
def ctx():
    pv3d.load(build_if_missing=True)
    c = pv3d.Context(device=0)
    yield c
    c.close()


def workloads():
    f = S.make_facade(seed=17, n=4, map_res=2048, n_buildings=20, n_trees=8, n_poles=4, floors=3, per_floor=8,
                      target_tris=8000, days=np.array([10, 80, 170, 260, 340]), radius=100.0)
    f.gen.string = (np.arange(f.gen.n_modules) // 4).astype(np.int32) * 7 + 3  # strings of 4 along each floor
    t = S.make_tracker(seed=9, n=4, map_res=1024, grid=(4, 3), terrain_n=64, spacing=1.5, n_pylons=2,
                       step_h=1.0, days=np.array([30, 172, 300]))   # strings: rows of 6 modules per table
    r = S.make_random_small(29, n_mods=9, n_steps=12, n=3, map_res=512)
    r.gen.string = np.array([5, 5, 5, 1, 1, 9, 9, 9, 9], np.int32)
    return [f, t, r]


@pytest.mark.parametrize("k", [0, 1, 2])
def test_string_power_and_energy(ctx, k):
    w = workloads()[k]
    gid = pv3d.load_workload(ctx, w)
    np.testing.assert_array_equal(ctx.string_ids(gid), np.unique(w.gen.string))
    g = run_gpu(ctx, gid, w, outputs=OUTS, chunk_steps=7)
    steps = np.arange(w.sun.n_steps)
    # 1. the string model on the GPU's own counts
    p_o, pu_o = oracle.string_power_from_counts(w, steps, g["cell_counts"].astype(np.int32))
    for got, ref in ((g["string_power"], p_o), (g["string_power_unshaded"], pu_o)):
        assert np.all(np.abs(got - ref) <= 1e-4 * np.maximum(np.abs(ref), 1.0) + 1e-3), np.abs(got - ref).max()
    # 2. energies: Kahan FP32 sums of the string powers
    dt = w.sun.dt_h.astype(np.float64)[:, None]
    lit = (w.sun.xyz[:, 2] > 0)[:, None]
    e64 = (g["string_power"].astype(np.float64) * dt * lit).sum(0)
    assert np.all(np.abs(g["string_energy"] - e64) <= 1e-6 * np.maximum(e64, 1.0))
    # 3. string losses in the oracle's envelope (masked samples forced lit / shaded)
    o = oracle.evaluate_workload(w)
    assert o["modules"].size == w.gen.n_modules
    lo, _ = oracle.string_power_from_counts(w, steps, oracle.popcount64(o["bits"] | o["mbits"]))
    hi, _ = oracle.string_power_from_counts(w, steps, oracle.popcount64(o["bits"] & ~o["mbits"]))
    eu = (pu_o * dt).sum(0)
    on = eu > 0
    l_g = 100 * (1 - g["string_energy"][on] / eu[on])
    l_min = 100 * (1 - (hi * dt).sum(0)[on] / eu[on])
    l_max = 100 * (1 - (lo * dt).sum(0)[on] / eu[on])
    assert np.all(l_g >= l_min - LOSS_PP) and np.all(l_g <= l_max + LOSS_PP), (l_min, l_g, l_max)
    # 4. a string never beats its modules' own maximum power points
    idx = np.searchsorted(np.unique(w.gen.string), w.gen.string)
    p_mod = np.zeros_like(g["string_power"])
    np.add.at(p_mod.T, idx, g["power"].T)
    assert np.all(g["string_power"] <= p_mod + 1e-3 + 1e-5 * p_mod)
    ctx.release(gid)


def test_one_module_per_string_is_the_module_model(ctx):
    w = S.make_random_small(31, n_mods=6, n_steps=10, n=3, map_res=512, tracked=True)
    w.gen.string = np.arange(w.gen.n_modules, dtype=np.int32)[::-1].copy()  # ids descending: order is by id
    gid = pv3d.load_workload(ctx, w)
    g = run_gpu(ctx, gid, w, outputs=OUTS)
    order = np.argsort(w.gen.string)
    np.testing.assert_allclose(g["string_power"], g["power"][:, order], rtol=1e-6, atol=1e-4)
    np.testing.assert_allclose(g["string_energy"], g["energy"][order], rtol=1e-6, atol=1e-4)
    ctx.release(gid)


def test_string_outputs_on_map_path_and_host(ctx):
    w = workloads()[2]
    gid = pv3d.load_workload(ctx, w)
    a = run_gpu(ctx, gid, w, outputs=OUTS)
    b = run_gpu(ctx, gid, w, outputs=OUTS, path=pv3d.PV3D_PATH_MAP)
    h = run_gpu(ctx, gid, w, outputs=OUTS, device=False)
    for k in ("string_power", "string_energy", "string_energy_unshaded"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
        np.testing.assert_array_equal(a[k], h[k], err_msg=k)
    # served requests produce them too, bit-identical to the evaluation alone
    rid, arr = ctx.submit(gid, n=w.n, map_res=w.map_res, outputs=("string_energy", "string_power"))
    assert ctx.poll(rid, timeout_ms=-1) == pv3d.PV3D_OK
    np.testing.assert_array_equal(arr["string_energy"].cpu().numpy(), a["string_energy"])
    np.testing.assert_array_equal(arr["string_power"].cpu().numpy(), a["string_power"])
    ctx.release(gid)


def test_parallel_strings(ctx):
    """Arrays of strings in parallel (one voltage per inverter input): per step
    the GPU's array power from its own counts equals the oracle's parallel
    model; one string per array is the string model; the array never beats
    its strings' own maxima; energies are the Kahan sums."""
    w = workloads()[0]
    w.gen.array = (w.gen.string // 14).astype(np.int32) * 5   # strings of 4 modules, arrays of two strings
    gid = pv3d.load_workload(ctx, w)
    np.testing.assert_array_equal(ctx.array_ids(gid), np.unique(w.gen.array))
    outs = OUTS + ("array_power", "array_power_unshaded", "array_energy", "array_energy_unshaded")
    g = run_gpu(ctx, gid, w, outputs=outs, chunk_steps=7)
    steps = np.arange(w.sun.n_steps)
    ap, apu = oracle.array_power_from_counts(w, steps, g["cell_counts"].astype(np.int32))
    for got, ref in ((g["array_power"], ap), (g["array_power_unshaded"], apu)):
        assert np.all(np.abs(got - ref) <= 1e-4 * np.maximum(np.abs(ref), 1.0) + 1e-3), np.abs(got - ref).max()
    _, str_array = oracle.array_index(w.gen)
    sp = np.zeros_like(g["array_power"])
    np.add.at(sp.T, str_array, g["string_power"].T)
    assert np.all(g["array_power"] <= sp + 1e-3 + 1e-5 * sp)
    dt = w.sun.dt_h.astype(np.float64)[:, None]
    lit = (w.sun.xyz[:, 2] > 0)[:, None]
    e64 = (g["array_power"].astype(np.float64) * dt * lit).sum(0)
    assert np.all(np.abs(g["array_energy"] - e64) <= 1e-6 * np.maximum(e64, 1.0))
    ctx.release(gid)
    w.gen.array = w.gen.string.copy()   # one string per array
    gid = pv3d.load_workload(ctx, w)
    g = run_gpu(ctx, gid, w, outputs=outs)
    np.testing.assert_allclose(g["array_power"], g["string_power"], rtol=1e-6, atol=1e-4)
    bad = w.gen.string.copy()
    bad_arr = np.arange(w.gen.n_modules, dtype=np.int32)   # modules of one string in different arrays
    w.gen.array = bad_arr
    with pytest.raises(pv3d.PV3DError):
        pv3d.load_workload(ctx, w)
    ctx.release(gid)
