"""Seeded synthetic inputs shaped like the paper's application cases (Section 3).

This module builds scenes (triangle soups), PV generators (module/cell grids,
bypass layouts, tracker pivots), sun tables and tracker poses.  It holds none
of the method's arithmetic: no light-space projection, no occlusion, no
reduction and no PV model.  Both the CUDA path and the FP64 oracle consume its
outputs, which are plain numpy arrays.

The paper's datasets (3D Warehouse models, Google Earth buildings, a surveyed
terrain) are not available, so each case is stood in for by a seeded
procedural scene of the same kind and size:

* ``tiny``     -- two 6x10-cell modules tilted 30 deg south at 40 N, one 2x2x3 m
                  box 3 m south, 24 hourly suns of one day (Section 2, Fig. 4 style).
* ``facade``   -- BIPV facade: 200 vertical modules among box buildings, cone
                  trees and lighting poles, ~50k triangles, hourly year
                  (Section 3.1 / 3.3 stand-in, 80,000-triangle scale of Section 4).
* ``tracker``  -- 500 two-axis trackers on a fractal heightmap with lattice pylons
                  and a distant ridge, quarter-hour year (Section 3.4 stand-in).

Sun positions use solar time with Cooper's declination and a spherical-astronomy
sun vector; irradiance uses the Meinel clear-sky beam formula with the
Kasten-Young air mass and DHI = 0.1 DNI (the paper allows a clear-sky model,
Section 2 step 4, without naming one).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

CELL_PITCH = 0.156  # m, 156 mm cells


# ---------------------------------------------------------------------------
# containers
# ---------------------------------------------------------------------------
@dataclass
class Scene:
    verts: np.ndarray  # (V, 3) float32, metres, ENU (x east, y north, z up)
    tris: np.ndarray   # (T, 3) int32

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


@dataclass
class Layout:
    cells_u: int
    cells_v: int
    n_sub: int
    cell_sub: np.ndarray  # (cells_v * cells_u,) int32, cell index c = cv * cells_u + cu


@dataclass
class Generator:
    origin: np.ndarray   # (M, 3) float32; tracker-local (relative to the pivot) when tracker >= 0
    u: np.ndarray        # (M, 3) float32 unit vector along increasing cell column cu
    v: np.ndarray        # (M, 3) float32 unit vector along increasing cell row cv
    cells_u: np.ndarray  # (M,) int32
    cells_v: np.ndarray  # (M,) int32
    pitch: np.ndarray    # (M,) float32
    layout: np.ndarray   # (M,) int32 index into layouts
    tracker: np.ndarray  # (M,) int32, -1 = fixed
    string: np.ndarray   # (M,) int32
    layouts: list = field(default_factory=list)
    pivots: np.ndarray = field(default_factory=lambda: np.zeros((0, 3), np.float32))
    array: np.ndarray | None = None  # (M,) int32 inverter input of the module's string (None: all 0)

    @property
    def n_modules(self) -> int:
        return int(self.origin.shape[0])

    @property
    def n_cells(self) -> int:
        return int((self.cells_u.astype(np.int64) * self.cells_v).sum())


@dataclass
class Sun:
    xyz: np.ndarray   # (N, 3) float64 unit vector toward the sun
    dni: np.ndarray   # (N,) float32 W/m^2
    dhi: np.ndarray   # (N,) float32 W/m^2
    dt_h: np.ndarray  # (N,) float32 hours

    @property
    def n_steps(self) -> int:
        return int(self.xyz.shape[0])


@dataclass
class Workload:
    name: str
    scene: Scene
    gen: Generator
    sun: Sun
    poses: np.ndarray | None  # (N, Nt, 2) float32 (azimuth, tilt) radians, or None
    n: int                    # samples per cell side (n x n per cell)
    map_res: int              # shadow-map side R

    @property
    def samples_per_step(self) -> int:
        return self.gen.n_cells * self.n * self.n

    def n_tests(self) -> int:
        """Sample tests over the steps whose sun is above the horizon."""
        return int((self.sun.xyz[:, 2] > 0).sum()) * self.samples_per_step


# ---------------------------------------------------------------------------
# sun table (input generation)
# ---------------------------------------------------------------------------
def declination_cooper(day: np.ndarray) -> np.ndarray:
    """Cooper (1969) declination in radians for day-of-year ``day`` (1..365)."""
    return np.radians(23.45) * np.sin(np.radians(360.0 * (284.0 + day) / 365.0))


def sun_vectors(lat_deg: float, day: np.ndarray, hour: np.ndarray) -> np.ndarray:
    """Unit ENU vector toward the sun at solar time ``hour`` (no equation of time)."""
    phi = math.radians(lat_deg)
    dec = declination_cooper(np.asarray(day, np.float64))
    h = np.radians(15.0 * (np.asarray(hour, np.float64) - 12.0))
    east = -np.cos(dec) * np.sin(h)
    north = np.sin(dec) * math.cos(phi) - np.cos(dec) * np.cos(h) * math.sin(phi)
    up = np.sin(dec) * math.sin(phi) + np.cos(dec) * np.cos(h) * math.cos(phi)
    s = np.stack([east, north, up], axis=-1)
    return s / np.linalg.norm(s, axis=-1, keepdims=True)


def clear_sky_dni(up: np.ndarray) -> np.ndarray:
    """Meinel & Meinel (1976) beam irradiance with Kasten-Young (1989) air mass."""
    up = np.clip(up, 1e-9, 1.0)
    zen = np.degrees(np.arccos(up))
    am = 1.0 / (up + 0.50572 * np.power(np.maximum(96.07995 - zen, 1e-6), -1.6364))
    return 1353.0 * np.power(0.7, np.power(am, 0.678))


def year_sun(lat_deg: float, step_h: float, daylight_only: bool = True,
             days: np.ndarray | None = None) -> Sun:
    if days is None:
        days = np.arange(1, 366)
    hours = np.arange(0.0, 24.0, step_h)
    dd, hh = np.meshgrid(days, hours, indexing="ij")
    s = sun_vectors(lat_deg, dd.ravel(), hh.ravel())
    if daylight_only:
        s = s[s[:, 2] > 0]
    dni = clear_sky_dni(s[:, 2]).astype(np.float32)
    dni[s[:, 2] <= 0] = 0
    return Sun(xyz=s.astype(np.float64), dni=dni, dhi=(0.1 * dni).astype(np.float32),
               dt_h=np.full(s.shape[0], step_h, np.float32))


def ideal_poses(sun: Sun, n_trackers: int, tilt_max_deg: float = 75.0) -> np.ndarray:
    """Two-axis tracker pose per step: face the sun's azimuth, tilt = zenith angle,
    clamped to ``tilt_max_deg``.  Returns (N, Nt, 2) float32 (azimuth, tilt) radians,
    azimuth on the compass (from north, clockwise)."""
    s = sun.xyz
    az = np.arctan2(s[:, 0], s[:, 1])
    tilt = np.minimum(np.arccos(np.clip(s[:, 2], -1, 1)), math.radians(tilt_max_deg))
    pose = np.stack([az, tilt], axis=-1).astype(np.float32)
    return np.repeat(pose[:, None, :], n_trackers, axis=1)


# ---------------------------------------------------------------------------
# geometry builders
# ---------------------------------------------------------------------------
class MeshBuilder:
    def __init__(self):
        self.v: list[np.ndarray] = []
        self.t: list[np.ndarray] = []
        self.nv = 0

    def add(self, verts, tris):
        verts = np.asarray(verts, np.float64).reshape(-1, 3)
        tris = np.asarray(tris, np.int64).reshape(-1, 3)
        self.v.append(verts)
        self.t.append(tris + self.nv)
        self.nv += verts.shape[0]

    def grid_quad(self, p0, eu, ev, nu, nv):
        """Planar quad p0 + a*eu + b*ev (a, b in [0,1]) split into nu x nv cells."""
        p0, eu, ev = (np.asarray(x, np.float64) for x in (p0, eu, ev))
        a = np.linspace(0, 1, nu + 1)
        b = np.linspace(0, 1, nv + 1)
        aa, bb = np.meshgrid(a, b, indexing="xy")
        verts = p0 + aa.ravel()[:, None] * eu + bb.ravel()[:, None] * ev
        idx = np.arange((nu + 1) * (nv + 1)).reshape(nv + 1, nu + 1)
        q00 = idx[:-1, :-1].ravel(); q10 = idx[:-1, 1:].ravel()
        q01 = idx[1:, :-1].ravel(); q11 = idx[1:, 1:].ravel()
        tris = np.concatenate([np.stack([q00, q10, q11], 1), np.stack([q00, q11, q01], 1)])
        self.add(verts, tris)

    def box(self, lo, hi, faces=("-x", "+x", "-y", "+y", "-z", "+z"), edge=None):
        lo = np.asarray(lo, np.float64); hi = np.asarray(hi, np.float64)
        d = hi - lo
        ex, ey, ez = np.eye(3)

        def n_of(length):
            return 1 if edge is None else max(1, int(round(length / edge)))
        spec = {
            "-x": (lo, ey * d[1], ez * d[2], d[1], d[2]),
            "+x": (lo + ex * d[0], ey * d[1], ez * d[2], d[1], d[2]),
            "-y": (lo, ex * d[0], ez * d[2], d[0], d[2]),
            "+y": (lo + ey * d[1], ex * d[0], ez * d[2], d[0], d[2]),
            "-z": (lo, ex * d[0], ey * d[1], d[0], d[1]),
            "+z": (lo + ez * d[2], ex * d[0], ey * d[1], d[0], d[1]),
        }
        for f in faces:
            p0, eu, ev, lu, lv = spec[f]
            self.grid_quad(p0, eu, ev, n_of(lu), n_of(lv))

    def beam(self, a, b, w):
        """Square-section member of width ``w`` from point a to point b (4 sides, 8 tris)."""
        a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
        ax = b - a
        ax_n = ax / np.linalg.norm(ax)
        ref = np.array([0.0, 0.0, 1.0]) if abs(ax_n[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
        e1 = np.cross(ax_n, ref); e1 /= np.linalg.norm(e1)
        e2 = np.cross(ax_n, e1)
        h = 0.5 * w
        ring = [(-h, -h), (h, -h), (h, h), (-h, h)]
        verts = [a + x * e1 + y * e2 for x, y in ring] + [b + x * e1 + y * e2 for x, y in ring]
        tris = []
        for k in range(4):
            k1 = (k + 1) % 4
            tris += [(k, k1, 4 + k1), (k, 4 + k1, 4 + k)]
        self.add(verts, tris)

    def cylinder(self, base, radius, height, seg):
        ang = np.linspace(0, 2 * np.pi, seg, endpoint=False)
        ring = np.stack([np.cos(ang) * radius, np.sin(ang) * radius, np.zeros(seg)], 1)
        base = np.asarray(base, np.float64)
        verts = np.concatenate([base + ring, base + ring + [0, 0, height]])
        tris = []
        for k in range(seg):
            k1 = (k + 1) % seg
            tris += [(k, k1, seg + k1), (k, seg + k1, seg + k)]
        self.add(verts, tris)

    def cone(self, base, radius, height, seg):
        """Side surface plus base disc of a cone (2*seg triangles)."""
        ang = np.linspace(0, 2 * np.pi, seg, endpoint=False)
        base = np.asarray(base, np.float64)
        ring = base + np.stack([np.cos(ang) * radius, np.sin(ang) * radius, np.zeros(seg)], 1)
        verts = np.concatenate([ring, [base + [0, 0, height]], [base]])
        apex, centre = seg, seg + 1
        tris = []
        for k in range(seg):
            k1 = (k + 1) % seg
            tris += [(k, k1, apex), (k1, k, centre)]
        self.add(verts, tris)

    def heightmap(self, x0, y0, spacing, h):
        ny, nx = h.shape
        xs = x0 + spacing * np.arange(nx)
        ys = y0 + spacing * np.arange(ny)
        xx, yy = np.meshgrid(xs, ys, indexing="xy")
        verts = np.stack([xx.ravel(), yy.ravel(), h.ravel()], 1)
        idx = np.arange(nx * ny).reshape(ny, nx)
        q00 = idx[:-1, :-1].ravel(); q10 = idx[:-1, 1:].ravel()
        q01 = idx[1:, :-1].ravel(); q11 = idx[1:, 1:].ravel()
        tris = np.concatenate([np.stack([q00, q10, q11], 1), np.stack([q00, q11, q01], 1)])
        self.add(verts, tris)

    def build(self) -> Scene:
        if not self.v:
            return Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32))
        return Scene(np.concatenate(self.v).astype(np.float32),
                     np.concatenate(self.t).astype(np.int32))


def standard_layout(cells_u: int, cells_v: int, n_sub: int) -> Layout:
    """Bypass substrings as equal groups of adjacent cell columns (cu), each
    running the full module height -- the usual 3-diode 60-cell wiring."""
    if cells_u % n_sub != 0:
        raise ValueError("cells_u must be a multiple of n_sub")
    cols = cells_u // n_sub
    cu = np.tile(np.arange(cells_u), cells_v)
    return Layout(cells_u, cells_v, n_sub, (cu // cols).astype(np.int32))


def _gen_from_lists(origins, us, vs, cu, cv, layout_ids, trackers, strings, layouts, pivots):
    m = len(origins)
    return Generator(
        origin=np.asarray(origins, np.float32).reshape(m, 3),
        u=np.asarray(us, np.float32).reshape(m, 3),
        v=np.asarray(vs, np.float32).reshape(m, 3),
        cells_u=np.full(m, cu, np.int32) if np.isscalar(cu) else np.asarray(cu, np.int32),
        cells_v=np.full(m, cv, np.int32) if np.isscalar(cv) else np.asarray(cv, np.int32),
        pitch=np.full(m, CELL_PITCH, np.float32),
        layout=np.asarray(layout_ids, np.int32),
        tracker=np.asarray(trackers, np.int32),
        string=np.asarray(strings, np.int32),
        layouts=layouts,
        pivots=np.asarray(pivots, np.float32).reshape(-1, 3),
    )


# ---------------------------------------------------------------------------
# the three single-scene cases
# ---------------------------------------------------------------------------
def make_tiny(day: int = 172, n: int = 4, map_res: int = 1024, seed: int = 0) -> Workload:
    """Two modules 6x10 cells, 30 deg tilt facing south, lat 40 N; a 2x2x3 m box
    whose centre is 3 m south of the modules; 24 hourly suns of one day."""
    del seed  # fully deterministic
    tilt = math.radians(30.0)
    u = (1.0, 0.0, 0.0)
    v = (0.0, math.cos(tilt), math.sin(tilt))
    w = 6 * CELL_PITCH
    origins = [(-w - 0.005, 0.0, 0.5), (0.005, 0.0, 0.5)]
    lay = standard_layout(6, 10, 3)
    gen = _gen_from_lists(origins, [u, u], [v, v], 6, 10, [0, 0], [-1, -1], [0, 0], [lay],
                          np.zeros((0, 3)))
    mb = MeshBuilder()
    mb.box((-1.0, -4.0, 0.0), (1.0, -2.0, 3.0))  # 12 triangles
    scene = mb.build()
    hours = np.arange(24, dtype=np.float64)
    s = sun_vectors(40.0, np.full(24, day), hours)
    sun = Sun(xyz=s, dni=np.full(24, 800.0, np.float32), dhi=np.full(24, 100.0, np.float32),
              dt_h=np.ones(24, np.float32))
    return Workload(f"tiny_day{day}", scene, gen, sun, None, n, map_res)


def _scatter_nonoverlap(rng, n, sampler, radius_of, existing=()):
    placed = list(existing)
    out = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > 20000:
            break  # crowded: keep the objects placed so far
        c, r = sampler(), None
        r = radius_of(c)
        if all(np.hypot(c[0] - q[0], c[1] - q[1]) > r + qr + 2.0 for q, qr in placed):
            placed.append((c, r))
            out.append(c)
    return out, placed


def make_facade(seed: int = 1, n: int = 8, map_res: int = 4096, n_buildings: int = 60,
                n_trees: int = 30, n_poles: int = 10, floors: int = 8, per_floor: int = 25,
                target_tris: int = 50000, step_h: float = 1.0, days=None,
                radius: float = 250.0) -> Workload:
    """BIPV facade: ``floors * per_floor`` vertical south-facing modules (6x10 cells,
    3 substrings) on the south face of an office block, seeded box buildings
    (8-40 m high) in the southern half-disc, cone trees and lighting poles."""
    rng = np.random.default_rng(seed)
    width = per_floor * 1.0 + 1.0
    height = floors * 3.0 + 0.5
    # generator: modules flush on the facade plane y = 0, normal -y
    u = (1.0, 0.0, 0.0)
    v = (0.0, 0.0, 1.0)
    origins = []
    for f in range(floors):
        for k in range(per_floor):
            origins.append((-0.5 * width + 0.5 + k * 1.0 + 0.032, 0.0, f * 3.0 + 0.7))
    m = len(origins)
    lay = standard_layout(6, 10, 3)
    gen = _gen_from_lists(origins, [u] * m, [v] * m, 6, 10, [0] * m, [-1] * m,
                          list(range(m)), [lay], np.zeros((0, 3)))

    # office block behind the facade (its south face is the module surface itself)
    mb = MeshBuilder()
    mb.box((-0.5 * width, 0.0, 0.0), (0.5 * width, 20.0, height), faces=("-x", "+x", "+y", "+z"),
           edge=3.0)

    # buildings in the southern half-disc
    def bsample():
        r = radius * math.sqrt(rng.uniform(0.04, 1.0))
        a = rng.uniform(math.pi, 2 * math.pi)
        return np.array([r * math.cos(a), r * math.sin(a) - 5.0])
    sizes = {}

    def brad(c):
        key = (float(c[0]), float(c[1]))
        if key not in sizes:
            sizes[key] = (rng.uniform(10, 28), rng.uniform(10, 28), rng.uniform(8, 40))
        sx, sy, _ = sizes[key]
        return 0.5 * math.hypot(sx, sy)
    block = [(np.array([0.0, 10.0]), 0.5 * math.hypot(width, 20.0) + 8.0)]
    centres, placed = _scatter_nonoverlap(rng, n_buildings, bsample, brad, block)
    dims = [sizes[(float(c[0]), float(c[1]))] for c in centres]
    # pick an edge length that brings the total near the target triangle count
    n_tree_tris = n_trees * (16 + 3 * 64)
    n_pole_tris = n_poles * 24
    budget = max(target_tris - n_tree_tris - n_pole_tris - 200, 12 * n_buildings)
    area = sum(2 * (sx + sy) * h + sx * sy for sx, sy, h in dims)
    edge = math.sqrt(2.0 * area / budget)
    for c, (sx, sy, h) in zip(centres, dims):
        lo = (c[0] - sx / 2, c[1] - sy / 2, 0.0)
        hi = (c[0] + sx / 2, c[1] + sy / 2, h)
        mb.box(lo, hi, faces=("-x", "+x", "-y", "+y", "+z"), edge=edge)

    # trees: trunk + three stacked 32-segment cones
    def tsample():
        r = rng.uniform(18.0, 120.0)
        a = rng.uniform(math.pi * 1.05, math.pi * 1.95)
        return np.array([r * math.cos(a), r * math.sin(a)])
    tree_c, placed = _scatter_nonoverlap(rng, n_trees, tsample, lambda c: 3.5, placed)
    for c in tree_c:
        hgt = rng.uniform(6.0, 14.0)
        rad = rng.uniform(2.0, 3.5)
        trunk_h = 0.25 * hgt
        mb.cylinder((c[0], c[1], 0.0), 0.25, trunk_h, 8)
        for k in range(3):
            z0 = trunk_h + k * 0.22 * hgt
            mb.cone((c[0], c[1], z0), rad * (1.0 - 0.22 * k), 0.45 * hgt, 32)

    # lighting poles along a street 12 m south of the facade
    for k in range(n_poles):
        x = -0.5 * width + (k + 0.5) * width / n_poles
        mb.beam((x, -12.0, 0.0), (x, -12.0, 8.0), 0.18)
        mb.beam((x, -12.0, 7.8), (x, -10.6, 7.8), 0.1)
        mb.box((x - 0.25, -10.9, 7.6), (x + 0.25, -10.3, 7.8), faces=("-x", "+x", "-y", "+y"))
    scene = mb.build()
    sun = year_sun(40.0, step_h, days=days)
    return Workload("facade", scene, gen, sun, None, n, map_res)


def fbm_heightmap(rng, size: int, relief: float, beta: float = 3.2) -> np.ndarray:
    """Fractional-Brownian-motion heightmap by spectral synthesis, scaled to +-relief."""
    kx = np.fft.fftfreq(size)[:, None]
    ky = np.fft.rfftfreq(size)[None, :]
    k = np.sqrt(kx * kx + ky * ky)
    k[0, 0] = 1.0
    amp = k ** (-beta / 2.0)
    amp[0, 0] = 0.0
    phase = rng.uniform(0, 2 * np.pi, amp.shape)
    spec = amp * (rng.standard_normal(amp.shape)) * np.exp(1j * phase)
    h = np.fft.irfft2(spec, s=(size, size))
    h -= h.mean()
    return relief * h / np.abs(h).max()


def make_tracker(seed: int = 2, n: int = 4, map_res: int = 8192, grid=(25, 20),
                 terrain_n: int = 512, spacing: float = 1.2, relief: float = 8.0,
                 n_pylons: int = 20, step_h: float = 0.25, days=None,
                 tilt_max_deg: float = 75.0, table=(6, 4), with_ridge: bool = True) -> Workload:
    """Two-axis tracker plant on uneven ground with lattice pylons and a ridge."""
    rng = np.random.default_rng(seed)
    size = (terrain_n - 1) * spacing
    x0 = y0 = -0.5 * size
    h = fbm_heightmap(rng, terrain_n, relief)

    def ground(x, y):
        fx = (x - x0) / spacing; fy = (y - y0) / spacing
        ix = int(np.clip(math.floor(fx), 0, terrain_n - 2)); iy = int(np.clip(math.floor(fy), 0, terrain_n - 2))
        ax = fx - ix; ay = fy - iy
        return ((1 - ax) * (1 - ay) * h[iy, ix] + ax * (1 - ay) * h[iy, ix + 1]
                + (1 - ax) * ay * h[iy + 1, ix] + ax * ay * h[iy + 1, ix + 1])

    mb = MeshBuilder()
    mb.heightmap(x0, y0, spacing, h)

    gx, gy = grid
    pitch_x = (size - 20.0) / gx
    pitch_y = (size - 20.0) / gy
    # table: table[0] modules across (x), table[1] modules up (y), portrait 6x12 cells
    mw, mh = 6 * CELL_PITCH, 12 * CELL_PITCH
    gap = 0.02
    tw = table[0] * mw + (table[0] - 1) * gap
    th = table[1] * mh + (table[1] - 1) * gap
    pivots = []
    for j in range(gy):
        for i in range(gx):
            px = x0 + 10.0 + (i + 0.5) * pitch_x + rng.uniform(-2.0, 2.0)
            py = y0 + 10.0 + (j + 0.5) * pitch_y + rng.uniform(-2.0, 2.0)
            pivots.append((px, py, ground(px, py) + 4.0))
    origins, trackers = [], []
    for t in range(len(pivots)):
        for r in range(table[1]):
            for c in range(table[0]):
                origins.append((-0.5 * tw + c * (mw + gap), -0.5 * th + r * (mh + gap), 0.0))
                trackers.append(t)
    m = len(origins)
    lay = standard_layout(6, 12, 3)
    gen = _gen_from_lists(origins, [(1.0, 0.0, 0.0)] * m, [(0.0, 1.0, 0.0)] * m, 6, 12,
                          [0] * m, trackers, [k // table[0] for k in range(m)], [lay], pivots)

    # lattice pylons along a north-south corridor between two tracker columns
    cx = x0 + 10.0 + (gx // 2) * pitch_x
    for k in range(n_pylons):
        py = y0 + 10.0 + (k + 1.0) * (size - 20.0) / (n_pylons + 1)
        _pylon(mb, (cx, py, ground(cx, py) - 0.5), rng)

    if with_ridge:
        # ridge ~150 m high, ~2 km east of the plant, running north-south
        nr_a, nr_b = 40, 8
        a = np.linspace(-1500.0, 1500.0, nr_a + 1)
        b = np.linspace(-400.0, 400.0, nr_b + 1)
        aa, bb = np.meshgrid(a, b, indexing="xy")
        zz = 150.0 * np.exp(-(bb / 180.0) ** 2) * (1.0 - (aa / 1700.0) ** 2)
        verts = np.stack([2000.0 + bb.ravel(), aa.ravel(), zz.ravel() - 5.0], 1)
        idx = np.arange((nr_a + 1) * (nr_b + 1)).reshape(nr_b + 1, nr_a + 1)
        q00 = idx[:-1, :-1].ravel(); q10 = idx[:-1, 1:].ravel()
        q01 = idx[1:, :-1].ravel(); q11 = idx[1:, 1:].ravel()
        mb.add(verts, np.concatenate([np.stack([q00, q10, q11], 1), np.stack([q00, q11, q01], 1)]))
    scene = mb.build()
    sun = year_sun(40.0, step_h, days=days)
    poses = ideal_poses(sun, len(pivots), tilt_max_deg)
    return Workload("tracker", scene, gen, sun, poses, n, map_res)


def _pylon(mb: MeshBuilder, base, rng, height: float = 30.0, levels: int = 14):
    """Lattice tower of thin square members (~2,000 triangles)."""
    bx, by, bz = base
    half0, half1 = 3.0, 0.9
    zs = np.linspace(0.0, height, levels + 1)

    def corner(k, z):
        s = half0 + (half1 - half0) * (z / height)
        sx = (-1, 1, 1, -1)[k]; sy = (-1, -1, 1, 1)[k]
        return np.array([bx + sx * s, by + sy * s, bz + z])
    for li in range(levels):
        z0, z1 = zs[li], zs[li + 1]
        for k in range(4):
            k1 = (k + 1) % 4
            mb.beam(corner(k, z0), corner(k, z1), 0.10)          # leg segment
            mb.beam(corner(k, z1), corner(k1, z1), 0.06)         # ring
            mb.beam(corner(k, z0), corner(k1, z1), 0.05)         # diagonal
            mb.beam(corner(k1, z0), corner(k, z1), 0.05)         # counter-diagonal
    # cross arms
    for za in (0.75 * height, 0.9 * height):
        mb.beam((bx - 8.0, by, bz + za), (bx + 8.0, by, bz + za), 0.12)
        mb.beam((bx - 8.0, by, bz + za), (bx - 0.5, by, bz + za + 2.0), 0.06)
        mb.beam((bx + 8.0, by, bz + za), (bx + 0.5, by, bz + za + 2.0), 0.06)
    del rng


# ---------------------------------------------------------------------------
# small random cases for parity tests
# ---------------------------------------------------------------------------
def make_random_small(seed: int, n_mods: int = 6, n_boxes: int = 5, n_steps: int = 12,
                      n: int = 3, map_res: int = 512, tracked: bool = False,
                      lat: float = 40.0) -> Workload:
    """A few modules (fixed rows or small trackers) among random boxes and poles,
    with suns spread over one year; sizes chosen so the oracle runs in seconds."""
    rng = np.random.default_rng(seed)
    mb = MeshBuilder()
    for _ in range(n_boxes):
        c = rng.uniform(-12, 12, 2)
        if np.hypot(*c) < 3.0:
            c = c * 3.0 / max(np.hypot(*c), 1e-3)
        sx, sy, hz = rng.uniform(0.5, 4.0), rng.uniform(0.5, 4.0), rng.uniform(1.0, 6.0)
        mb.box((c[0] - sx / 2, c[1] - sy / 2, 0.0), (c[0] + sx / 2, c[1] + sy / 2, hz),
               faces=("-x", "+x", "-y", "+y", "+z"), edge=rng.choice([None, 1.0]))
    for _ in range(2):
        c = rng.uniform(-6, 6, 2)
        mb.beam((c[0], c[1], 0.0), (c[0], c[1], rng.uniform(3.0, 6.0)), rng.uniform(0.05, 0.3))
    scene = mb.build()
    cu, cv = 6, int(rng.choice([8, 10, 12]))
    lay = standard_layout(cu, cv, 3)
    origins, us, vs, trk = [], [], [], []
    pivots = []
    if tracked:
        for k in range(n_mods):
            pivots.append((rng.uniform(-5, 5), rng.uniform(-5, 5), rng.uniform(1.5, 3.0)))
            origins.append((-0.5 * cu * CELL_PITCH, -0.5 * cv * CELL_PITCH, 0.0))
            us.append((1.0, 0.0, 0.0)); vs.append((0.0, 1.0, 0.0)); trk.append(k)
    else:
        tilt = math.radians(rng.uniform(0.0, 60.0))
        az = math.radians(rng.uniform(120.0, 240.0))
        # U horizontal, V up the slope; normal faces compass azimuth az
        uh = np.array([-math.cos(az), math.sin(az), 0.0])
        down = np.array([math.sin(az), math.cos(az), 0.0])
        vv = -down * math.cos(tilt) + np.array([0, 0, 1.0]) * math.sin(tilt)
        for k in range(n_mods):
            row, col = divmod(k, 3)
            base = np.array([0.0, 0.0, 0.4 + rng.uniform(0, 0.3)]) + uh * (col - 1.5) * (cu * CELL_PITCH + 0.02) \
                - down * row * 3.5
            origins.append(tuple(base)); us.append(tuple(uh)); vs.append(tuple(vv)); trk.append(-1)
    gen = _gen_from_lists(origins, us, vs, cu, cv, [0] * n_mods, trk, list(range(n_mods)), [lay],
                          np.asarray(pivots).reshape(-1, 3))
    # suns: random days and hours in daylight, plus some low-sun steps
    s_list = []
    while len(s_list) < n_steps:
        d = rng.integers(1, 366); hr = rng.uniform(4.0, 20.0)
        s = sun_vectors(lat, np.array([d]), np.array([hr]))[0]
        if s[2] > 0.03:
            s_list.append(s)
    s = np.array(s_list)
    dni = clear_sky_dni(s[:, 2]).astype(np.float32)
    sun = Sun(xyz=s, dni=dni, dhi=(0.1 * dni).astype(np.float32), dt_h=np.ones(len(s), np.float32))
    poses = ideal_poses(sun, len(pivots), 70.0) if tracked else None
    return Workload(f"random{seed}{'_trk' if tracked else ''}", scene, gen, sun, poses, n, map_res)


def make_canopy(seed: int, tiny_modules: bool = False, n_steps: int = 8, n: int = 3, map_res: int = 256,
                cells: int = 30, holes: float = 0.4, lat: float = 40.0) -> Workload:
    """A finely triangulated canopy with random holes (a pergola or a tree
    crown stand-in) over either four tilted modules or a field of 1-cell
    modules 0.2 m apart.  On a coarse map one raster tile holds hundreds of
    the canopy's triangles, or dozens of receiver modules: the workloads the
    tile kernels hand from one warp per tile to one block per tile."""
    rng = np.random.default_rng(seed)
    mb = MeshBuilder()
    side = 3.0
    p0 = np.array([-side / 2, -side / 2, 2.5])
    eu, ev = np.array([side, 0.0, 0.15]), np.array([0.0, side, 0.0])
    a = np.linspace(0, 1, cells + 1)
    aa, bb = np.meshgrid(a, a, indexing="xy")
    verts = p0 + aa.ravel()[:, None] * eu + bb.ravel()[:, None] * ev
    idx = np.arange((cells + 1) ** 2).reshape(cells + 1, cells + 1)
    keep = rng.random((cells, cells)) >= holes
    q00, q10 = idx[:-1, :-1][keep], idx[:-1, 1:][keep]
    q01, q11 = idx[1:, :-1][keep], idx[1:, 1:][keep]
    mb.add(verts, np.concatenate([np.stack([q00, q10, q11], 1), np.stack([q00, q11, q01], 1)]))
    mb.beam((-1.6, -1.6, 0.0), (-1.6, -1.6, 2.6), 0.1)
    mb.beam((1.6, 1.6, 0.0), (1.6, 1.6, 2.6), 0.1)
    scene = mb.build()
    if tiny_modules:
        lay = Layout(1, 1, 1, np.zeros(1, np.int32))
        g = np.arange(-1.4, 1.41, 0.2)
        xx, yy = np.meshgrid(g, g, indexing="xy")
        origins = [(x, y, 0.5) for x, y in zip(xx.ravel(), yy.ravel())]
        m = len(origins)
        gen = _gen_from_lists(origins, [(1.0, 0.0, 0.0)] * m, [(0.0, 1.0, 0.0)] * m, 1, 1, [0] * m, [-1] * m,
                              list(range(m)), [lay], np.zeros((0, 3)))
    else:
        cu, cv = 6, 10
        lay = standard_layout(cu, cv, 3)
        tilt = math.radians(20.0)
        vv = (0.0, math.cos(tilt), math.sin(tilt))
        origins = [(-1.0 + 1.0 * (k % 2) - 0.47, -1.4 + 1.5 * (k // 2), 0.6) for k in range(4)]
        gen = _gen_from_lists(origins, [(1.0, 0.0, 0.0)] * 4, [vv] * 4, cu, cv, [0] * 4, [-1] * 4, list(range(4)),
                              [lay], np.zeros((0, 3)))
    s_list = []
    while len(s_list) < n_steps:
        d = rng.integers(1, 366); hr = rng.uniform(8.0, 16.0)
        sv = sun_vectors(lat, np.array([d]), np.array([hr]))[0]
        if sv[2] > 0.3:
            s_list.append(sv)
    sv = np.array(s_list)
    dni = clear_sky_dni(sv[:, 2]).astype(np.float32)
    sun = Sun(xyz=sv, dni=dni, dhi=(0.1 * dni).astype(np.float32), dt_h=np.ones(len(sv), np.float32))
    return Workload(f"canopy{seed}{'_tiny' if tiny_modules else ''}", scene, gen, sun, None, n, map_res)


def make_config(name: str, **kw) -> Workload:
    if name in ("tiny", "cfg1"):
        return make_tiny(**kw)
    if name in ("facade", "cfg2"):
        return make_facade(**kw)
    if name in ("tracker", "cfg3"):
        return make_tracker(**kw)
    raise KeyError(name)


# ---------------------------------------------------------------------------
# many scenes of uneven size (batched and served workloads)
# ---------------------------------------------------------------------------
def _pow2_at_least(x: float, lo: int, hi: int) -> int:
    r = lo
    while r < x and r < hi:
        r *= 2
    return r


def make_mixed_scene(rng, tris_target: int, mods_target: int, lat: float, n_steps: int, n: int = 4) -> Workload:
    """A facade-like or tracker-like scene with about ``tris_target`` triangles,
    ``mods_target`` modules, suns of ``n_steps`` consecutive daylight hours of a
    year at latitude ``lat``."""
    seed = int(rng.integers(1 << 30))
    if rng.random() < 0.5:
        per_floor = int(np.clip(round(math.sqrt(mods_target * 3)), 2, 60))
        floors = int(np.clip(math.ceil(mods_target / per_floor), 1, 40))
        nb = int(np.clip(tris_target // 700, 2, 60))
        w = make_facade(seed=seed, n=n, map_res=1024, n_buildings=nb, n_trees=int(np.clip(nb // 2, 1, 30)),
                        n_poles=int(np.clip(nb // 4, 1, 10)), floors=floors, per_floor=per_floor,
                        target_tris=tris_target,
                        radius=float(max(2.5 * (per_floor + 1), 15.0 * math.sqrt(nb) + 40.0 + per_floor)))
    else:
        trackers = max(1, int(math.ceil(mods_target / 24)))
        gx = int(math.ceil(math.sqrt(trackers * 1.25)))
        gy = int(math.ceil(trackers / gx))
        terrain_n = int(np.clip(round(math.sqrt(max(tris_target, 200) / 2.0)), 8, 512))
        size = 25.0 * max(gx, gy) + 30
        spacing = size / (terrain_n - 1)
        w = make_tracker(seed=seed, n=n, map_res=1024, grid=(gx, gy), terrain_n=terrain_n, spacing=spacing,
                         n_pylons=int(rng.integers(0, 3)), step_h=1.0, with_ridge=bool(rng.random() < 0.3))
    full = year_sun(lat, 1.0)
    k = int(min(n_steps, full.n_steps))
    b = int(rng.integers(0, full.n_steps - k + 1))
    w.sun = Sun(xyz=full.xyz[b:b + k], dni=full.dni[b:b + k], dhi=full.dhi[b:b + k], dt_h=full.dt_h[b:b + k])
    if w.poses is not None:
        w.poses = ideal_poses(w.sun, w.gen.pivots.shape[0])
    # light window finer than half the sample spacing, within 512..4096
    pts = w.gen.pivots if w.gen.pivots.shape[0] else w.gen.origin
    ext = float(np.ptp(pts, axis=0).max() + 10.0)
    w.map_res = _pow2_at_least(2.0 * ext / (CELL_PITCH / n), 512, 4096)
    w.name = f"mixed{seed}"
    return w


def make_batch(seed: int = 4, n_scenes: int = 256, tris=(1e3, 2e5), mods=(10, 2000), lat=(0.0, 60.0),
               steps=(100, 4400), n: int = 4) -> list:
    """``n_scenes`` scenes of uneven size: triangles and modules log-uniform,
    latitude uniform, sun steps uniform (the batched workload)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_scenes):
        t = int(math.exp(rng.uniform(math.log(tris[0]), math.log(tris[1]))))
        m = int(math.exp(rng.uniform(math.log(mods[0]), math.log(mods[1]))))
        out.append(make_mixed_scene(rng, t, m, float(rng.uniform(*lat)), int(rng.integers(steps[0], steps[1] + 1)),
                                    n=n))
    return out
