"""Pins of the FP64 oracle against what geometry and the paper fix (no GPU).

Each test checks the oracle against something other than itself: a closed
form (pole shadow length, convex-obstacle shadow polygon, infinite-sheds
row-to-row fraction, PV-model special cases), brute force, or an invariant of
the method (Robledo et al., Section 2 steps 3-4).
"""
import math
import numpy as np
import pytest
from scipy.spatial import ConvexHull

import oracle
from paper_1410_5780_gb300 import scenes as S

def sun_from(az_deg, el_deg):
    az, el = math.radians(az_deg), math.radians(el_deg)
    return np.array([math.sin(az) * math.cos(el), math.cos(az) * math.cos(el), math.sin(el)])


def one_sun(s, dni=800.0, dhi=100.0):
    s = np.asarray(s, np.float64).reshape(-1, 3)
    k = s.shape[0]
    return S.Sun(xyz=s, dni=np.full(k, dni, np.float32), dhi=np.full(k, dhi, np.float32),
                 dt_h=np.ones(k, np.float32))


def flat_gen(origins, u, v, cells_u, cells_v, n_sub=1, pitch=S.CELL_PITCH):
    m = len(origins)
    lay = S.Layout(cells_u, cells_v, n_sub,
                   (np.tile(np.arange(cells_u), cells_v) // (cells_u // n_sub)).astype(np.int32))
    g = S._gen_from_lists(origins, [u] * m, [v] * m, cells_u, cells_v, [0] * m, [-1] * m,
                          list(range(m)), [lay], np.zeros((0, 3)))
    g.pitch = np.full(m, pitch, np.float32)
    return g


# ---------------------------------------------------------------------------
# ray test: BVH against brute force
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bvh_rays_equal_brute_force(seed):
    rng = np.random.default_rng(seed)
    nt = 300
    c = rng.uniform(-5, 5, (nt, 1, 3))
    verts = (c + rng.normal(0, 0.8, (nt, 3, 3))).reshape(-1, 3).astype(np.float32)
    tris = np.arange(3 * nt, dtype=np.int32).reshape(nt, 3)
    sc = oracle.OracleScene(verts, tris)
    o = rng.uniform(-6, 6, (4000, 3))
    d = rng.normal(size=(4000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    a = sc.rays(o, d, brute=False)
    b = sc.rays(o, d, brute=True)
    assert a.sum() > 200 and (~a).sum() > 200
    assert np.array_equal(a, b)


@pytest.mark.parametrize("seed,tracked", [(11, False), (12, True), (13, False)])
def test_bvh_evaluate_equals_brute_force(seed, tracked):
    w = S.make_random_small(seed, n_mods=4, n_steps=5, n=3, tracked=tracked)
    a = oracle.evaluate_workload(w, brute=False)
    b = oracle.evaluate_workload(w, brute=True)
    assert np.array_equal(a["bits"], b["bits"])
    assert np.array_equal(a["mbits"], b["mbits"])
    assert np.array_equal(a["power"], b["power"])


# ---------------------------------------------------------------------------
# closed form: the shadow of a pole of height h has length h / tan(elevation)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("el_deg", [15.0, 30.0, 47.0, 70.0])
def test_pole_shadow_length(el_deg):
    w_pole, h = 0.3, 4.0
    mb = S.MeshBuilder()
    mb.box((-w_pole / 2, -w_pole / 2, 0.0), (w_pole / 2, w_pole / 2, h))
    scene = mb.build()
    # horizontal strip north of the pole, sun due south
    pitch = 0.05
    cu, cv = 16, 400
    origin = (-cu * pitch / 2, w_pole / 2 + 0.01, 0.0)
    gen = flat_gen([origin], (1, 0, 0), (0, 1, 0), cu, cv, pitch=pitch)
    sun = one_sun(sun_from(180.0, el_deg))
    n = 2
    r = oracle.evaluate(scene, gen, sun, None, n, 1024)
    flags = oracle.unpack_bits(r["bits"][0], n)  # [cells, 4]
    xyz = oracle.samples(gen, None, 0, 0, n).reshape(cv * cu, n * n, 3)
    x, y = xyz[..., 0], xyz[..., 1]
    length = h / math.tan(math.radians(el_deg))
    inside = (np.abs(x) < w_pole / 2 - 1e-3) & (y < w_pole / 2 + length - 1e-3)
    outside = (np.abs(x) > w_pole / 2 + 1e-3) | (y > w_pole / 2 + length + 1e-3)
    assert inside.sum() > 0
    assert flags[inside].all()
    assert not flags[outside].any()


# ---------------------------------------------------------------------------
# closed form: a convex obstacle in front of a plane shades exactly the convex
# hull of its vertices projected onto the plane along the sun direction
# ---------------------------------------------------------------------------
def _hull_contains(poly2d, pts, margin):
    hull = ConvexHull(poly2d)
    eq = hull.equations  # a.x + b.y + c <= 0 inside, with (a, b) unit
    dist = pts @ eq[:, :2].T + eq[:, 2]
    inside = (dist < -margin).all(axis=1)
    outside = (dist > margin).any(axis=1)
    return inside, outside


@pytest.mark.parametrize("day,hours", [(355, range(8, 17)), (20, range(9, 16))])
def test_convex_obstacle_shadow_polygon(day, hours):
    w = S.make_tiny(day=day)
    s_all = S.sun_vectors(40.0, np.full(len(hours), day), np.asarray(list(hours), float))
    sun = one_sun(s_all)
    n = 4
    r = oracle.evaluate(w.scene, w.gen, sun, None, n, 1024)
    box = w.scene.verts.astype(np.float64)[np.unique(w.scene.tris)]
    checked = 0
    for m in range(w.gen.n_modules):
        o = w.gen.origin[m].astype(np.float64)
        u = w.gen.u[m].astype(np.float64)
        v = w.gen.v[m].astype(np.float64)
        nrm = np.cross(u, v); nrm /= np.linalg.norm(nrm)
        xyz = oracle.samples(w.gen, None, 0, m, n)
        loc = np.stack([(xyz - o) @ u, (xyz - o) @ v], 1)
        c0 = 60 * m
        for si in range(len(s_all)):
            s = s_all[si]
            flags = oracle.unpack_bits(r["bits"][si, c0:c0 + 60], n).reshape(-1)
            if nrm @ s <= 0:
                continue
            hgt = (box - o) @ nrm
            assert (hgt > 0).all()  # the box lies wholly in front of the module plane
            proj = box - np.outer(hgt / (nrm @ s), s)
            poly = np.stack([(proj - o) @ u, (proj - o) @ v], 1)
            inside, outside = _hull_contains(poly, loc, 1e-6)
            assert flags[inside].all()
            assert not flags[outside].any()
            checked += int(inside.sum())
    assert checked > 100


# ---------------------------------------------------------------------------
# closed form: infinite sheds, row-to-row shaded fraction
#   f = clamp(1 - (d/L) sin(a_p) / sin(a_p + beta), 0, 1)
# ---------------------------------------------------------------------------
def sheds_fraction(beta, d_over_l, alpha_p):
    return min(1.0, max(0.0, 1.0 - d_over_l * math.sin(alpha_p) / math.sin(alpha_p + beta)))


def test_sheds_helper_worked_example():
    # beta = 30 deg, d/L = 2, alpha_p = 20 deg: 1 - 2 sin20 / sin50 = 0.1070
    assert abs(sheds_fraction(math.radians(30), 2.0, math.radians(20)) - 0.1070) < 5e-5


@pytest.mark.parametrize("beta_deg,d_over_l,el_deg,az_deg",
                         [(30.0, 2.0, 20.0, 180.0), (25.0, 1.8, 14.0, 180.0),
                          (35.0, 2.5, 18.0, 205.0), (20.0, 2.2, 40.0, 180.0)])
def test_infinite_sheds_fraction(beta_deg, d_over_l, el_deg, az_deg):
    beta = math.radians(beta_deg)
    cu, cv, pitch, n = 240, 8, S.CELL_PITCH, 4
    L = cv * pitch
    d = d_over_l * L
    u = (1.0, 0.0, 0.0)
    v = (0.0, math.cos(beta), math.sin(beta))
    rows = 5
    origins = [(-cu * pitch / 2, k * d, 0.0) for k in range(rows)]
    gen = flat_gen(origins, u, v, cu, cv, pitch=pitch)
    scene = S.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32))
    s = sun_from(az_deg, el_deg)
    sun = one_sun(s)
    r = oracle.evaluate(scene, gen, sun, None, n, 2048, modules=[2], want_mask=False)
    # profile angle of the sun seen across the rows (rows face south, az 180)
    alpha_p = math.atan(math.tan(math.radians(el_deg)) / math.cos(math.radians(az_deg - 180.0)))
    f_exp = sheds_fraction(beta, d_over_l, alpha_p)
    flags = oracle.unpack_bits(r["bits"][0], n).reshape(cv, cu, n, n)  # [cv, cu, j, i]
    mid = flags[:, cu // 2 - 20: cu // 2 + 20]
    # slant position of each sample row along the module
    b = (np.arange(cv)[:, None] + (np.arange(n)[None, :] + 0.5) / n) * pitch  # [cv, j]
    b_shadow = f_exp * L
    expect = np.broadcast_to((b < b_shadow)[:, None, :, None], mid.shape)
    near = np.broadcast_to((np.abs(b - b_shadow) < 1e-4)[:, None, :, None], mid.shape)
    assert np.array_equal(mid[~near], expect[~near])
    frac = mid.mean()
    assert abs(frac - f_exp) <= 1.0 / (cv * n) + 1e-12


# ---------------------------------------------------------------------------
# PV model closed forms (series-current-limited bypass-diode model)
# ---------------------------------------------------------------------------
def test_pv_unshaded_closed_form():
    lay = S.standard_layout(6, 10, 3)
    for G in (100.0, 523.5, 1000.0):
        p = oracle.module_pmpp(np.full(60, G), lay.cell_sub, 3)
        assert abs(p - oracle.I_REF * G / 1000.0 * 60 * oracle.V_CELL) < 1e-9


def test_pv_one_shaded_cell_closed_form():
    lay = S.standard_layout(6, 10, 3)
    vk = 20 * oracle.V_CELL
    for g_full, g_diff in [(900.0, 100.0), (900.0, 400.0), (300.0, 250.0), (800.0, 0.0)]:
        g = np.full(60, g_full)
        g[0] = g_diff
        i_full = oracle.I_REF * g_full / 1000.0
        i_diff = oracle.I_REF * g_diff / 1000.0
        expect = max(i_full * (2 * vk - oracle.V_DIODE), i_diff * 3 * vk)
        assert abs(oracle.module_pmpp(g, lay.cell_sub, 3) - expect) < 1e-9


def test_pv_two_substrings_hand_case():
    # substrings at 9, 4.5 and 2.7 A (G 1000, 500, 300): candidates
    # 9 A * (10 - 0.5 - 0.5) = 81 W; 4.5 A * (20 - 0.5) = 87.75 W; 2.7 A * 30 = 81 W
    lay = S.standard_layout(6, 10, 3)
    g = np.full(60, 1000.0)
    sub = lay.cell_sub
    g[np.flatnonzero(sub == 1)[3]] = 500.0
    g[np.flatnonzero(sub == 2)[7]] = 300.0
    assert abs(oracle.module_pmpp(g, sub, 3) - 87.75) < 1e-9


def test_pv_monotone_in_irradiance():
    rng = np.random.default_rng(5)
    lay = S.standard_layout(6, 12, 3)
    for _ in range(200):
        g = rng.uniform(0, 1000, 72)
        p0 = oracle.module_pmpp(g, lay.cell_sub, 3)
        g2 = g.copy()
        k = rng.integers(72)
        g2[k] *= rng.uniform(0, 1)
        assert oracle.module_pmpp(g2, lay.cell_sub, 3) <= p0 + 1e-12


def test_pv_mpp_is_max_over_current_scan():
    """The maximum over the substring currents equals a fine scan of P(I)."""
    rng = np.random.default_rng(6)
    lay = S.standard_layout(6, 10, 3)
    for _ in range(30):
        g = rng.uniform(50, 1000, 60)
        ic = oracle.I_REF * g / 1000.0
        ik = np.array([ic[lay.cell_sub == k].min() for k in range(3)])
        grid = np.linspace(0, ik.max(), 20001)
        volts = np.where(ik[None, :] >= grid[:, None], 20 * oracle.V_CELL, -oracle.V_DIODE).sum(1)
        scan = max(0.0, float((grid * volts).max()))
        p = oracle.module_pmpp(g, lay.cell_sub, 3)
        assert p >= scan - 1e-9
        assert p <= scan + ik.max() / 20000 * 60 * oracle.V_CELL + 1e-9


def _substrings(g, cell_sub, n_sub):
    ic = oracle.I_REF * np.asarray(g, float) / 1000.0
    ik = np.array([ic[cell_sub == k].min() for k in range(n_sub)])
    vk = np.array([(cell_sub == k).sum() * oracle.V_CELL for k in range(n_sub)])
    return ik, vk


def test_string_two_modules_closed_forms():
    """A series string of two 60-cell, 3-substring modules (Fig. 2 wiring): the
    unshaded string delivers the two modules' power; with one beam-shaded cell
    in one module, the best of bypassing its substring (5 substrings at full
    current, one diode drop) and limiting the whole string to the shaded
    cell's current (6 substrings)."""
    lay = S.standard_layout(6, 10, 3)
    vk = 20 * oracle.V_CELL
    for g_full, g_diff in [(900.0, 100.0), (900.0, 700.0), (300.0, 250.0), (800.0, 0.0)]:
        a = np.full(60, g_full)
        ik_a, vk_a = _substrings(a, lay.cell_sub, 3)
        p2 = oracle.series_pmpp(np.r_[ik_a, ik_a], np.r_[vk_a, vk_a])
        assert abs(p2 - 2 * oracle.I_REF * g_full / 1000.0 * 60 * oracle.V_CELL) < 1e-9
        b = a.copy()
        b[0] = g_diff
        ik_b, vk_b = _substrings(b, lay.cell_sub, 3)
        i_full, i_diff = oracle.I_REF * g_full / 1000.0, oracle.I_REF * g_diff / 1000.0
        expect = max(i_full * (5 * vk - oracle.V_DIODE), i_diff * 6 * vk)
        assert abs(oracle.series_pmpp(np.r_[ik_a, ik_b], np.r_[vk_a, vk_b]) - expect) < 1e-9


def test_string_of_one_module_is_the_module():
    rng = np.random.default_rng(8)
    lay = S.standard_layout(6, 12, 3)
    for _ in range(100):
        g = rng.uniform(0, 1000, 72)
        ik, vk = _substrings(g, lay.cell_sub, 3)
        assert abs(oracle.series_pmpp(ik, vk) - oracle.module_pmpp(g, lay.cell_sub, 3)) < 1e-9


def test_string_mpp_is_max_over_current_scan_and_below_module_mppt():
    """The string's maximum over substring currents equals a fine scan of
    P(I); and it never exceeds the sum of its modules' own maxima (one
    tracker per module can only do better than one per string)."""
    rng = np.random.default_rng(9)
    lay = S.standard_layout(6, 10, 3)
    for _ in range(30):
        gs = [rng.uniform(50, 1000, 60) for _ in range(int(rng.integers(2, 6)))]
        subs = [_substrings(g, lay.cell_sub, 3) for g in gs]
        ik = np.concatenate([a for a, _ in subs]); vk = np.concatenate([b for _, b in subs])
        grid = np.linspace(0, ik.max(), 40001)
        volts = np.where(ik[None, :] >= grid[:, None], vk[None, :], -oracle.V_DIODE).sum(1)
        scan = max(0.0, float((grid * volts).max()))
        p = oracle.series_pmpp(ik, vk)
        assert scan - 1e-9 <= p <= scan + ik.max() / 40000 * vk.sum() + 1e-9
        assert p <= sum(oracle.module_pmpp(g, lay.cell_sub, 3) for g in gs) + 1e-9


def test_parallel_strings_closed_forms_and_scan():
    """Strings in parallel at one voltage: one string is the series model; k
    identical strings give k times its power; a fine voltage scan (each
    string's current = the largest current on a fine grid whose string voltage
    still reaches V) agrees; the array never beats its strings' own maxima."""
    lay = S.standard_layout(6, 10, 3)
    rng = np.random.default_rng(12)
    for _ in range(20):
        strings = []
        for _ in range(int(rng.integers(1, 5))):
            gs = [rng.uniform(50, 1000, 60) for _ in range(int(rng.integers(1, 4)))]
            subs = [_substrings(g, lay.cell_sub, 3) for g in gs]
            strings.append((np.concatenate([a for a, _ in subs]), np.concatenate([b for _, b in subs])))
        p = oracle.parallel_pmpp(strings)
        if len(strings) == 1:
            assert abs(p - oracle.series_pmpp(*strings[0])) < 1e-9
        assert abs(oracle.parallel_pmpp([strings[0]] * 3) - 3 * oracle.series_pmpp(*strings[0])) < 1e-9
        assert p <= sum(oracle.series_pmpp(a, b) for a, b in strings) + 1e-9
        # brute force: voltage scan, currents on a fine grid
        imax = max(a.max() for a, _ in strings)
        igrid = np.linspace(0, imax, 4001)
        curves = []
        for a, b in strings:
            v_of_i = np.where(a[None, :] >= igrid[:, None], b[None, :], -oracle.V_DIODE).sum(1)  # non-increasing
            curves.append(v_of_i)
        vmax = max(c.max() for c in curves)
        best = 0.0
        for V in np.linspace(0, vmax, 3001):
            cur = 0.0
            for c in curves:
                ok = np.flatnonzero(c >= V)
                cur += igrid[ok[-1]] if ok.size else 0.0
            best = max(best, V * cur)
        assert best - 1e-9 <= p <= best + (imax / 4000 + 0) * vmax * len(strings) + vmax / 3000 * imax * len(strings) + 1e-9


def test_string_power_from_counts_matches_modules_and_strings():
    """String powers from shaded counts: with every module its own string they
    are the module powers; grouped into strings they follow series_pmpp of the
    members' substrings; zero counts give the unshaded string power."""
    w = S.make_random_small(61, n_mods=6, n_steps=5, n=2)
    steps = np.arange(w.sun.n_steps)
    rng = np.random.default_rng(3)
    C = int((w.gen.cells_u * w.gen.cells_v).sum())
    counts = rng.integers(0, w.n * w.n + 1, (steps.size, C)).astype(np.int32)
    p_mod = oracle.power_from_counts(w, steps, np.arange(w.gen.n_modules), counts)
    w.gen.string = np.arange(w.gen.n_modules, dtype=np.int32)
    p, pu = oracle.string_power_from_counts(w, steps, counts)
    np.testing.assert_allclose(p, p_mod, rtol=1e-12, atol=1e-12)
    pu_mod = oracle.power_from_counts(w, steps, np.arange(w.gen.n_modules), np.zeros_like(counts))
    np.testing.assert_allclose(pu, pu_mod, rtol=1e-12, atol=1e-12)
    w.gen.string = np.array([7, 7, 3, 3, 3, 9], np.int32)   # strings 3, 7, 9 in ascending order
    p, pu = oracle.string_power_from_counts(w, steps, counts)
    assert p.shape == (steps.size, 3)
    assert np.all(p <= p_mod[:, [2, 3, 4]].sum(1)[:, None] * [1, 0, 0] + p_mod[:, [0, 1]].sum(1)[:, None] * [0, 1, 0]
                  + p_mod[:, [5]].sum(1)[:, None] * [0, 0, 1] + 1e-9)
    np.testing.assert_allclose(p[:, 2], p_mod[:, 5], rtol=1e-12, atol=1e-12)
    # arrays of strings in parallel: one array per string is the string model
    w.gen.array = np.array([0, 0, 1, 1, 1, 2], np.int32)
    ap, apu = oracle.array_power_from_counts(w, steps, counts)
    np.testing.assert_allclose(ap, p[:, [1, 0, 2]], rtol=1e-12, atol=1e-12)  # strings 3, 7, 9 -> arrays 1, 0, 2
    w.gen.array = np.array([4, 4, 4, 4, 4, 4], np.int32)
    ap, apu = oracle.array_power_from_counts(w, steps, counts)
    assert ap.shape == (steps.size, 1) and np.all(ap[:, 0] <= p.sum(1) + 1e-9)


def test_sun_table_closed_forms():
    """Noon elevation 90 - lat + delta (delta = 0 at the equinox day 81 of
    Cooper's formula, 23.45 sin(449.75 deg) at day 172), a 12-hour day at the
    equinox and 2 acos(-tan(lat) tan(delta)) / 15 hours otherwise, morning and
    afternoon mirror images, unit vectors."""
    for lat in (0.0, 23.0, 40.0, 52.5, -33.0):
        xyz, dni, dhi = oracle.sun_table(lat, 81, 1, 0.25, daylight_only=False)
        noon = xyz[48]
        assert abs(math.degrees(math.asin(noon[2])) - (90.0 - abs(lat))) < 1e-9
        np.testing.assert_allclose(np.linalg.norm(xyz, axis=1), 1.0, atol=1e-14)
        np.testing.assert_allclose(xyz[47 - np.arange(40)][:, [1, 2]], xyz[49 + np.arange(40)][:, [1, 2]], atol=1e-14)
        np.testing.assert_allclose(xyz[47 - np.arange(40)][:, 0], -xyz[49 + np.arange(40)][:, 0], atol=1e-14)
    d172 = math.radians(23.45 * math.sin(math.radians(360.0 * 456 / 365)))
    xyz, _, _ = oracle.sun_table(40.0, 172, 1, 1.0, daylight_only=False)
    assert abs(math.degrees(math.asin(xyz[12, 2])) - (50.0 + math.degrees(d172))) < 1e-9
    assert abs(math.degrees(math.asin(xyz[12, 2])) - 73.45) < 0.01
    # day length from the sunrise hour angle, counted on a fine grid
    for lat, day in ((40.0, 172), (40.0, 355), (60.0, 100)):
        dec = math.radians(23.45 * math.sin(math.radians(360.0 * (284 + day) / 365)))
        hours = 2 * math.degrees(math.acos(-math.tan(math.radians(lat)) * math.tan(dec))) / 15.0
        xyz, _, _ = oracle.sun_table(lat, day, 1, 0.01, daylight_only=True)
        assert abs(xyz.shape[0] * 0.01 - hours) <= 0.02


def test_sun_table_irradiance_published_values():
    """Meinel's beam at air mass 1 is 1353 * 0.7 = 947.1 W/m^2 (Kasten & Young
    give 0.9997 at the zenith); at 60 and 80 degrees of zenith their air mass
    lies just under the plane-parallel 1/cos z (2 and 5.76); night steps carry
    no irradiance; DHI = 0.1 DNI; the beam rises with the sun."""
    step = 1.0 / 3.0
    xyz, dni, dhi = oracle.sun_table(0.0, 81, 1, step, daylight_only=False)
    # equator at the equinox: the zenith angle equals |hour angle|
    am = (np.log(np.maximum(dni, 1e-300) / 1353.0) / math.log(0.7)) ** (1 / 0.678)
    noon, h8, h6_40 = 36, 24, 20           # solar hours 12, 8, 6:40 -> zenith 0, 60, 80 deg
    assert abs(dni[noon] - 947.1) < 0.4 and abs(am[noon] - 0.9997) < 3e-4
    assert 1.98 < am[h8] < 2.0
    assert 5.5 < am[h6_40] < 1.0 / math.cos(math.radians(80.0))
    assert np.all(dni[xyz[:, 2] <= 0] == 0) and np.all(dhi == 0.1 * dni)
    assert np.all(np.diff(dni[19:37]) > 0)


def test_heat_map_bins():
    """Bins by compass azimuth and zenith; energies and counts add up; night
    steps are left out."""
    s = np.array([[0.0, 1.0, 0.0001], [1.0, 0.0, 1.0], [0.0, -1.0, 1.0], [-1.0, 0.0, 0.2], [0.3, 0.2, -0.5]])
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    p = np.array([1.0, 2.0, 3.0, 4.0, 5.0]); pu = p + 1; dt = np.full(5, 0.5)
    e, eu, cnt = oracle.heat_map(s, p, pu, dt, 4, 3)
    assert cnt.sum() == 4 and abs(e.sum() - 0.5 * 10.0) < 1e-12 and abs(eu.sum() - 0.5 * 14.0) < 1e-12
    assert cnt[2, 0] == 1          # north at the horizon: azimuth 0, zenith ~90 (last bin)
    assert cnt[1, 1] == 1          # east at 45 deg zenith: azimuth 90
    assert cnt[1, 2] == 1          # south at 45 deg zenith: azimuth 180
    assert cnt[2, 3] == 1          # west, low


def test_sky_patches_cover_the_hemisphere():
    """The patches' solid angles add to 2 pi; the cosine-weighted sum
    approximates the projected hemisphere pi; the patch directions are unit
    vectors above the horizon."""
    for rings, sectors in ((9, 36), (18, 72), (3, 8)):
        xyz, dom = oracle.sky_patches(rings, sectors)
        assert abs(dom.sum() - 2 * math.pi) < 1e-12
        assert abs((dom * xyz[:, 2]).sum() - math.pi) < 1.05 / rings ** 2  # midpoint rule, O(1/rings^2)
        np.testing.assert_allclose(np.linalg.norm(xyz, axis=1), 1.0, atol=1e-14)
        assert xyz[:, 2].min() > 0


def _wall_workload(h, d, n=2):
    """A horizontal 1-cell module at the origin and a 400 m long wall of height
    h at distance d to its north."""
    mb = S.MeshBuilder()
    mb.grid_quad((-200.0, d, 0.0), (400.0, 0.0, 0.0), (0.0, 0.0, h), 40, 1)
    lay = S.Layout(1, 1, 1, np.zeros(1, np.int32))
    gen = S._gen_from_lists([(-0.078, -0.078, 0.0)], [(1.0, 0.0, 0.0)], [(0.0, 1.0, 0.0)], 1, 1, [0], [-1], [0],
                            [lay], np.zeros((0, 3)))
    sun = S.Sun(xyz=np.array([[0.0, 0.0, 1.0]]), dni=np.ones(1, np.float32), dhi=np.ones(1, np.float32),
                dt_h=np.ones(1, np.float32))
    return S.Workload("wall", mb.build(), gen, sun, None, n, 256)


@pytest.mark.parametrize("h,d", [(3.0, 3.0), (10.0, 4.0), (2.0, 8.0)])
def test_diffuse_shade_of_a_long_wall_closed_form(h, d):
    """A horizontal element beside an infinitely long wall of height h at
    distance d sees the wall over the fraction (1 - d / sqrt(d^2 + h^2)) / 2
    of its cosine-weighted sky (the two-dimensional view factor of a strip,
    Hottel's crossed strings); the oracle's patch quadrature gets it within
    0.01."""
    w = _wall_workload(h, d)
    xyz, _ = oracle.sky_patches(18, 72)
    wp = S.Workload(w.name, w.scene, w.gen, S.Sun(xyz=xyz, dni=np.ones(len(xyz), np.float32),
                                                  dhi=np.zeros(len(xyz), np.float32),
                                                  dt_h=np.ones(len(xyz), np.float32)), None, w.n, w.map_res)
    o = oracle.evaluate(wp.scene, wp.gen, wp.sun, None, wp.n, wp.map_res, want_mask=False)
    f = oracle.diffuse_shade_fractions(wp, 18, 72, o["counts"], np.array([[0.0, 0.0, 1.0]]))
    expect = 0.5 * (1 - d / math.hypot(d, h))
    assert abs(f[0] - expect) < 0.01, (f[0], expect)
    f0 = oracle.diffuse_shade_fractions(wp, 18, 72, np.zeros_like(o["counts"]), np.array([[0.0, 0.0, 1.0]]))
    assert f0[0] == 0.0


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
def test_no_obstacles_zero_loss():
    w = S.make_tiny(day=355)
    empty = S.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32))
    r = oracle.evaluate(empty, w.gen, w.sun, None, w.n, w.map_res)
    assert r["counts"].sum() == 0
    assert np.array_equal(r["power"], r["power_unshaded"])
    assert np.array_equal(r["energy"], r["energy_unshaded"])


def test_sun_below_horizon_zero():
    w = S.make_tiny(day=355)
    r = oracle.evaluate_workload(w)
    night = w.sun.xyz[:, 2] <= 0
    assert night.sum() > 0
    assert (r["power"][night] == 0).all() and (r["power_unshaded"][night] == 0).all()
    assert (r["counts"][night] == 0).all() and (r["delta"][night] == 0).all()


@pytest.mark.parametrize("seed", [21, 22])
def test_adding_occluder_never_reduces_loss(seed):
    base = S.make_random_small(seed, n_mods=4, n_steps=8, n=3)
    extra = S.MeshBuilder()
    rng = np.random.default_rng(seed + 100)
    for _ in range(4):
        c = rng.uniform(-6, 6, 2)
        extra.box((c[0] - 1, c[1] - 1, 0), (c[0] + 1, c[1] + 1, rng.uniform(2, 6)))
    ex = extra.build()
    verts = np.concatenate([base.scene.verts, ex.verts])
    tris = np.concatenate([base.scene.tris, ex.tris + base.scene.verts.shape[0]])
    more = S.Scene(verts, tris)
    a = oracle.evaluate_workload(base, want_mask=False)
    b = oracle.evaluate(more, base.gen, base.sun, base.poses, base.n, base.map_res, want_mask=False)
    assert ((a["bits"] & ~b["bits"]) == 0).all()
    assert (b["power"] <= a["power"] + 1e-12).all()
    assert (b["counts"].sum() > a["counts"].sum())


def test_fractions_are_multiples_of_one_over_n2():
    w = S.make_random_small(31, n_mods=3, n_steps=4, n=3)
    r = oracle.evaluate_workload(w)
    bits = oracle.unpack_bits(r["bits"], 3)
    assert np.array_equal(bits.sum(-1), r["counts"])


# ---------------------------------------------------------------------------
# parity mask: every sample whose exact answer changes within the texel-centre
# radius around it must be masked
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed,tracked", [(41, False), (42, True)])
def test_mask_covers_every_ambiguous_sample(seed, tracked):
    w = S.make_random_small(seed, n_mods=3, n_steps=4, n=3, map_res=256, tracked=tracked)
    r = oracle.evaluate_workload(w)
    n = w.n
    for si in range(w.sun.n_steps):
        s = w.sun.xyz[si]
        delta = r["delta"][si]
        # scene + all module quads, for the perturbed exact rays
        for e, m in enumerate(r["modules"]):
            nrm = oracle.module_normal(w.gen, w.poses, si, m)
            if nrm @ s <= math.cos(math.radians(89)):
                continue
            quads_v, quads_t = [], []
            for m2 in range(w.gen.n_modules):
                if m2 == m:
                    continue
                xyz2 = _module_corners(w, si, m2)
                base = len(quads_v) * 4
                quads_v.append(xyz2)
                quads_t += [(base, base + 1, base + 2), (base, base + 2, base + 3)]
            verts = np.concatenate([w.scene.verts.astype(np.float64)] + quads_v).astype(np.float32)
            tris = np.concatenate([w.scene.tris, np.asarray(quads_t, np.int32).reshape(-1, 3)
                                   + w.scene.verts.shape[0]]).astype(np.int32)
            sc = oracle.OracleScene(verts, tris)
            xyz = oracle.samples(w.gen, w.poses, si, m, n)
            c0 = int(np.concatenate([[0], np.cumsum(r["cells_per_module"])])[e])
            nc = int(r["cells_per_module"][e])
            flags = oracle.unpack_bits(r["bits"][si, c0:c0 + nc], n).reshape(-1)
            masked = oracle.unpack_bits(r["mbits"][si, c0:c0 + nc], n).reshape(-1)
            # points on the module plane whose projections lie within 0.7 texel
            lu = np.array([s[1], -s[0], 0.0]); lu /= np.linalg.norm(lu)
            lv = np.cross(s, lu)
            t_u = lu - s * (nrm @ lu) / (nrm @ s)   # plane vector projecting onto lu
            t_v = lv - s * (nrm @ lv) / (nrm @ s)
            ang = np.linspace(0, 2 * np.pi, 16, endpoint=False)
            offs = [(0.0, 0.0)] + [(0.7 * delta * math.cos(a_), 0.7 * delta * math.sin(a_)) for a_ in ang] \
                + [(0.35 * delta * math.cos(a_), 0.35 * delta * math.sin(a_)) for a_ in ang[::2]]
            res = []
            for du, dv in offs:
                q = xyz + du * t_u + dv * t_v
                res.append(sc.rays(q, np.broadcast_to(s, q.shape), t_min=1e-9 * 100))
            res = np.stack(res)
            assert np.array_equal(res[0], flags)
            ambiguous = (res != res[0]).any(0)
            assert not (ambiguous & ~masked).any(), (si, m, np.flatnonzero(ambiguous & ~masked))
    # the mask must leave most samples checkable
    assert r["mbits"].size and _popcount(r["mbits"]) < 0.3 * r["mbits"].size * n * n


def _popcount(a):
    return int(sum(bin(int(x)).count("1") for x in a.ravel()))


def _module_corners(w, step, m):
    xyz = oracle.samples(w.gen, w.poses, step, m, 1)  # cell centres
    cu, cv = int(w.gen.cells_u[m]), int(w.gen.cells_v[m])
    p = float(w.gen.pitch[m])
    c = xyz.reshape(cv, cu, 3)
    du = (c[0, 1] - c[0, 0]) if cu > 1 else None
    dv = (c[1, 0] - c[0, 0]) if cv > 1 else None
    eu = du / np.linalg.norm(du) * p
    ev = dv / np.linalg.norm(dv) * p
    o = c[0, 0] - 0.5 * eu - 0.5 * ev
    return np.stack([o, o + cu * eu, o + cu * eu + cv * ev, o + cv * ev])


# ---------------------------------------------------------------------------
# samples, poses and the light window
# ---------------------------------------------------------------------------
def test_samples_tile_each_cell():
    w = S.make_tiny()
    for n in (1, 3, 4):
        xyz = oracle.samples(w.gen, None, 0, 1, n).reshape(10, 6, n * n, 3)
        o, u, v = (w.gen.origin[1].astype(float), w.gen.u[1].astype(float), w.gen.v[1].astype(float))
        p = float(w.gen.pitch[1])
        cen = xyz.mean(2)
        cv, cu = np.meshgrid(np.arange(10), np.arange(6), indexing="ij")
        exp = o + ((cu + 0.5) * p)[..., None] * u + ((cv + 0.5) * p)[..., None] * v
        assert np.allclose(cen, exp, atol=1e-6)
        a = (xyz - o) @ u
        b = (xyz - o) @ v
        assert (a > cu[..., None] * p).all() and (a < (cu[..., None] + 1) * p).all()
        assert (b > cv[..., None] * p).all() and (b < (cv[..., None] + 1) * p).all()


def test_tracker_pose_normal_closed_form():
    w = S.make_random_small(7, n_mods=3, n_steps=6, tracked=True)
    for st in range(w.sun.n_steps):
        for m in range(w.gen.n_modules):
            az, tilt = w.poses[st, w.gen.tracker[m]].astype(np.float64)
            exp = np.array([math.sin(tilt) * math.sin(az), math.sin(tilt) * math.cos(az), math.cos(tilt)])
            got = oracle.module_normal(w.gen, w.poses, st, m)
            assert np.allclose(got, exp, atol=1e-6)
            s = w.sun.xyz[st]
            if math.degrees(math.acos(s[2])) < 69.9:  # pose not clamped: faces the sun
                assert got @ s > 1 - 1e-6


def test_texel_size_closed_forms():
    a = 2.0
    gen = flat_gen([(-1.0, -1.0, 0.0)], (1, 0, 0), (0, 1, 0), 10, 10, pitch=a / 10)
    empty = S.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32))
    R = 512
    for el in (90.0, 60.0, 25.0):
        r = oracle.evaluate(empty, gen, one_sun(sun_from(180.0, el)), None, 1, R, want_mask=False)
        assert abs(r["delta"][0] / (a / (R - 2)) - 1) < 1e-7  # float32 pitch
    # vertical facade W x H facing south, sun due south: extent max(W, H cos el)
    W, H = 3.0, 6.0
    gen = flat_gen([(0.0, 0.0, 0.0)], (1, 0, 0), (0, 0, 1), 10, 20, pitch=0.3)
    for el in (10.0, 45.0, 70.0):
        r = oracle.evaluate(empty, gen, one_sun(sun_from(180.0, el)), None, 1, R, want_mask=False)
        assert abs(r["delta"][0] / (max(W, H * math.cos(math.radians(el))) / (R - 2)) - 1) < 1e-7


# ---------------------------------------------------------------------------
# closed form: per-cell beam irradiation lost to shading (Section 2 step 4:
# beam removed from shaded areas, summed over the year)
# ---------------------------------------------------------------------------
def test_cell_beam_loss_straight_edge_closed_form():
    """A horizontal module (4 x 2 cells of 0.2 m, 4 x 4 samples) under a
    horizontal plate at height h = 1 m that covers x <= x_e = 1 m.  With the
    sun s = (sin z, 0, cos z) a sample at x is shaded iff x <= x_e - tan z, so
    each step's shadow edge is a straight line across the module; the steps
    put it through the middle of a cell column, past the module, before it,
    and one sun is below the horizon.  Per cell the oracle's beam loss must
    be sum_k DNI_k cos z_k dt_k f_k, with f_k the cell's share of samples left
    of the edge (DNI, cos and dt differ per step, so a dropped or swapped
    factor changes the sum)."""
    pitch, cu, cv, n = 0.2, 4, 2, 4
    gen = flat_gen([(0.0, 0.0, 0.0)], (1, 0, 0), (0, 1, 0), cu, cv, pitch=pitch)
    x_e, h = 1.0, 1.0
    verts = np.array([[-20.0, -20.0, h], [x_e, -20.0, h], [x_e, 20.0, h], [-20.0, 20.0, h]], np.float32)
    scene = S.Scene(verts, np.array([[0, 1, 2], [0, 2, 3]], np.int32))
    x_s = np.array([0.30, 0.90, 0.50, -0.10])          # shadow edge on the module per lit step
    tan_z = x_e - x_s
    z = np.arctan(tan_z)
    lit = np.stack([np.sin(z), np.zeros(4), np.cos(z)], 1)
    night = np.array([[0.8, 0.0, -0.6]])
    xyz = np.concatenate([lit[:2], night, lit[2:]])
    dni = np.array([700.0, 820.0, 450.0, 910.0, 640.0], np.float32)
    dt = np.array([1.0, 0.25, 1.0, 0.5, 1.0], np.float32)
    sun = S.Sun(xyz=xyz, dni=dni, dhi=np.full(5, 90.0, np.float32), dt_h=dt)
    r = oracle.evaluate(scene, gen, sun, None, n, 1024)
    # hand values: shaded sample columns per cell column for each edge
    #   x_s = 0.3: cell column 0 all 4, column 1 two of 4 (x = 0.225, 0.275), others none
    #   x_s = 0.9: all;  x_s = 0.5: columns 0, 1 all, column 2 two of 4;  x_s = -0.1: none
    f_col = {0.30: [1.0, 0.5, 0.0, 0.0], 0.90: [1.0, 1.0, 1.0, 1.0], 0.50: [1.0, 1.0, 0.5, 0.0],
             -0.10: [0.0, 0.0, 0.0, 0.0]}
    lit_rows = [0, 1, 3, 4]
    exp_col = np.zeros(cu)
    for k, xs in zip(lit_rows, x_s):
        cos_z = float(xyz[k, 2])
        exp_col += float(dni[k]) * cos_z * float(dt[k]) * np.array(f_col[round(float(xs), 2)])
    exp = np.tile(exp_col, cv)  # cells numbered cv * cells_u + cu
    assert np.allclose(r["cell_beam_loss"], exp, rtol=1e-12, atol=1e-9), (r["cell_beam_loss"], exp)
    # the fully shaded column equals the full beam over the lit steps; the
    # half-shaded cells half of their step's beam
    full = sum(float(dni[k]) * float(xyz[k, 2]) * float(dt[k]) for k in lit_rows[:3])
    assert abs(r["cell_beam_loss"][0] - full) < 1e-9
    assert abs(r["cell_beam_loss"][1] - (0.5 * 700.0 * float(xyz[0, 2]) + 820.0 * 0.25 * float(xyz[1, 2])
                                         + 910.0 * 0.5 * float(xyz[3, 2]))) < 1e-9


# ---------------------------------------------------------------------------
# closed form: a tracked module turns about its tracker's pivot
# ---------------------------------------------------------------------------
def test_tracker_pivot_cell_centres_closed_form():
    """One module in tracker-local coordinates (cells 2 x 1 of 0.3 m, origin
    (-0.3, -0.2, 0.05), axes x and y) on a tracker whose pivot is at
    (10, -3, 2).  For right-angle poses the rotation is a signed permutation
    of the axes, written here by hand: at tilt 0 facing south the module is
    only translated by the pivot; at tilt 90 deg facing south (az 180) local
    (x, y, z) -> (x, -z, y); facing east (az 90) -> (z, x, y); facing west
    (az 270) -> (-z, -x, y); at tilt 0 facing east -> (-y, x, z).  The cell
    centres (one sample per cell) must be the pivot plus the mapped local
    centre -- a pose about the origin instead of the pivot, or a dropped or
    misplaced pivot, fails."""
    g = flat_gen([(-0.3, -0.2, 0.05)], (1, 0, 0), (0, 1, 0), 2, 1, pitch=0.3)
    g.tracker = np.zeros(1, np.int32)
    g.pivots = np.array([[10.0, -3.0, 2.0]], np.float32)
    piv = np.array([10.0, -3.0, 2.0])
    local = np.array([[-0.15, -0.05, 0.05], [0.15, -0.05, 0.05]])  # cell centres, tracker-local
    cases = [
        (180.0, 0.0, lambda x, y, z: (x, y, z)),
        (180.0, 90.0, lambda x, y, z: (x, -z, y)),
        (90.0, 90.0, lambda x, y, z: (z, x, y)),
        (270.0, 90.0, lambda x, y, z: (-z, -x, y)),
        (90.0, 0.0, lambda x, y, z: (-y, x, z)),
    ]
    poses = np.array([[[math.radians(az), math.radians(t)]] for az, t, _ in cases], np.float32)
    for st, (az, t, f) in enumerate(cases):
        got = oracle.samples(g, poses, st, 0, 1)
        exp = np.array([piv + np.array(f(*c)) for c in local])
        assert np.allclose(got, exp, atol=2e-6), (az, t, got, exp)
        nrm = oracle.module_normal(g, poses, st, 0)
        assert np.allclose(nrm, np.array(f(0.0, 0.0, 1.0)), atol=1e-6)


def test_cell_beam_loss_from_counts_matches_the_evaluation():
    """The counts-based beam loss (used for the GPU envelope) equals the
    oracle's own per-cell sums on its own counts."""
    for w in (S.make_tiny(day=355), S.make_random_small(31, n_mods=4, n_steps=8, n=3, tracked=True)):
        o = oracle.evaluate_workload(w, want_mask=False)
        b = oracle.cell_beam_loss_from_counts(w, o["steps"], o["modules"], o["counts"], o["cos_inc"])
        assert o["cell_beam_loss"].max() > 0
        assert np.allclose(b, o["cell_beam_loss"], rtol=1e-12, atol=1e-9)


# ---------------------------------------------------------------------------
# diffuse shading of tracked modules: pose bins and the posed sky view
# ---------------------------------------------------------------------------
def test_pose_bins_hand_values():
    """Pose bins: azimuth sectors of [0, 360) deg (wrapped), tilt bands of
    [0, 90] deg (clamped), bin = band * sectors + sector, centre poses in the
    middle of both ranges -- values written out by hand."""
    d = math.radians
    poses = np.array([[d(10), d(5)], [d(-10), d(5)], [d(95), d(46)], [d(360 + 185), d(90)], [d(270), d(-3)]])
    b, az_c, tilt_c = oracle.pose_bins(poses, 4, 2)
    assert list(b) == [0, 3, 5, 6, 3]
    assert np.allclose(np.degrees(az_c[[0, 3, 5, 6]]), [45, 315, 135, 225])
    assert np.allclose(np.degrees(tilt_c[[0, 3, 5, 6]]), [22.5, 22.5, 67.5, 67.5])


def test_tracked_sky_view_equals_fixed_module_at_the_bin_pose():
    """A tracked module's diffuse fraction at pose bin (az 90, tilt 45 deg)
    equals that of a fixed module placed by hand where that pose puts it:
    R = Rz(pi - az) Rx(tilt) maps the local axes x -> (0, 1, 0) and y ->
    (-cos 45, 0, sin 45) (facing east, tilted 45 deg), the origin to
    pivot + R o.  The fixed path is pinned by the long wall's view factor."""
    mb = S.MeshBuilder()
    mb.grid_quad((3.0, -100.0, 0.0), (0.0, 200.0, 0.0), (0.0, 0.0, 6.0), 20, 1)   # wall 3 m east, 6 m high
    mb.box((-4.0, -2.0, 0.0), (-3.0, 2.0, 2.5))
    scene = mb.build()
    lay = S.Layout(3, 2, 1, np.zeros(6, np.int32))
    o_loc = np.array([-0.234, -0.156, 0.0])
    piv = np.array([0.5, 0.2, 2.0])
    g_trk = S._gen_from_lists([tuple(o_loc)], [(1.0, 0.0, 0.0)], [(0.0, 1.0, 0.0)], 3, 2, [0], [0], [0], [lay],
                              piv[None, :])
    c = math.cos(math.radians(45.0))
    u_w, v_w = np.array([0.0, 1.0, 0.0]), np.array([-c, 0.0, c])
    o_w = piv + o_loc[0] * u_w + o_loc[1] * v_w
    g_fix = S._gen_from_lists([tuple(o_w)], [tuple(u_w)], [tuple(v_w)], 3, 2, [0], [-1], [0], [lay], np.zeros((0, 3)))
    sun1 = S.Sun(xyz=np.array([[0.0, 0.0, 1.0]]), dni=np.ones(1, np.float32), dhi=np.ones(1, np.float32),
                 dt_h=np.ones(1, np.float32))
    poses = np.array([[[math.radians(100.0), math.radians(50.0)]]], np.float32)   # falls in bin (90, 45)
    w_trk = S.Workload("trk", scene, g_trk, sun1, poses, 3, 512)
    f_trk, _, step_bin = oracle.tracked_diffuse_fractions(w_trk, 6, 24, 2, 1, 3, 512, want_mask=False)
    assert list(step_bin) == [0] and list(f_trk) == [0]
    rings, sectors = 6, 24
    xyz, _ = oracle.sky_patches(rings, sectors)
    sun = S.Sun(xyz=xyz, dni=np.ones(len(xyz), np.float32), dhi=np.zeros(len(xyz), np.float32),
                dt_h=np.ones(len(xyz), np.float32))
    o = oracle.evaluate(scene, g_fix, sun, None, 3, 512, want_mask=False)
    nrm = np.repeat(np.cross(u_w, v_w)[None, :], 6, 0)
    f_fix = oracle.diffuse_shade_fractions(S.Workload("fix", scene, g_fix, sun, None, 3, 512), rings, sectors,
                                           o["counts"], nrm)
    assert f_fix.max() > 0.05  # the wall hides part of the east-facing module's sky
    assert np.allclose(f_trk[0], f_fix, atol=1e-12), (f_trk[0], f_fix)
