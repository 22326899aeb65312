"""FP64 CPU oracle for the 3DPV shadow-sample path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never calls it.  It
shares no code with the CUDA library: it is plain C (``pv3d_oracle.c``) built
with gcc, plus this ctypes wrapper.

``evaluate`` computes, for chosen sun steps and modules (Robledo et al.,
Section 2, steps 2-4):
  * per sample: shaded iff the exact FP64 ray toward the sun meets a triangle
    other than the sample's own module (Moller-Trumbore over a BVH);
  * per sample (optional): the parity mask -- the one-texel shadow-map answer is
    ambiguous there (see the C file's header);
  * per cell: shaded count; per module: MPP power shaded/unshaded with the
    series-current-limited bypass-diode model; energies over the steps.

``string_power_from_counts`` applies the same electrical model to series
strings of modules (one current and one maximum power point per string).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pv3d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

I_REF = 9.0      # A at 1000 W/m^2
V_CELL = 0.5     # V per cell at the operating point
V_DIODE = 0.5    # V across a conducting bypass diode


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu99", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.pv3d_oracle_scene_create.restype = P
            lib.pv3d_oracle_scene_create.argtypes = [P, C.c_int64, P, C.c_int64]
            lib.pv3d_oracle_scene_destroy.argtypes = [P]
            lib.pv3d_oracle_series_pmpp.restype = C.c_double
            lib.pv3d_oracle_series_pmpp.argtypes = [C.c_int32, P, P, C.c_double]
            lib.pv3d_oracle_module_pmpp.restype = C.c_double
            lib.pv3d_oracle_module_pmpp.argtypes = [C.c_int32, P, P, C.c_int32, C.c_double,
                                                    C.c_double, C.c_double]
            lib.pv3d_oracle_evaluate.restype = C.c_int
            lib.pv3d_oracle_evaluate.argtypes = (
                [P, C.c_int32, P, P, P, P, P, C.c_int32, P, P, P, P, P, P,
                 C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double,
                 P, C.c_int64, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
                + [P] * 10)
            lib.pv3d_oracle_samples.restype = C.c_int
            lib.pv3d_oracle_samples.argtypes = [C.c_int32, P, P, C.c_int32, P, P, C.c_int64,
                                                C.c_int32, C.c_int32, P]
            lib.pv3d_oracle_module_normal.restype = C.c_int
            lib.pv3d_oracle_module_normal.argtypes = [C.c_int32, P, P, C.c_int32, P, P, C.c_int64,
                                                      C.c_int32, P]
            lib.pv3d_oracle_power_from_counts.restype = C.c_int
            lib.pv3d_oracle_power_from_counts.argtypes = (
                [C.c_int32, P, P, P, P, P, C.c_int32, P, P, P, P, P, C.c_int32, C.c_double, C.c_double,
                 C.c_double, P, C.c_int64, P, C.c_int32, P, P])
            lib.pv3d_oracle_string_power_from_counts.argtypes = (
                [C.c_int32, P, P, P, P, P, C.c_int32, P, P, P, P, P, C.c_int32, C.c_double, C.c_double,
                 C.c_double, P, C.c_int64, P, C.c_int32, P, P, P, P, C.c_int32, P, P])
            lib.pv3d_oracle_parallel_pmpp.restype = C.c_double
            lib.pv3d_oracle_parallel_pmpp.argtypes = [C.c_int32, P, P, P, C.c_double]
            lib.pv3d_oracle_sun_table.restype = C.c_int64
            lib.pv3d_oracle_sun_table.argtypes = [C.c_double, C.c_int32, C.c_int32, C.c_double, C.c_int32,
                                                  C.c_double, P, P, P]
            lib.pv3d_oracle_rays.restype = C.c_int
            lib.pv3d_oracle_rays.argtypes = [P, P, P, C.c_int64, C.c_double, C.c_int32, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class OracleScene:
    """A triangle soup held by the oracle (FP64 copy plus BVH)."""

    def __init__(self, verts: np.ndarray, tris: np.ndarray):
        self.lib = _load()
        self.verts = np.ascontiguousarray(verts, np.float32)
        self.tris = np.ascontiguousarray(tris, np.int32)
        self.h = self.lib.pv3d_oracle_scene_create(_ptr(self.verts), self.verts.shape[0],
                                                   _ptr(self.tris), self.tris.shape[0])

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.pv3d_oracle_scene_destroy(self.h)
            self.h = None

    def rays(self, o: np.ndarray, d: np.ndarray, t_min: float = 1e-9, brute: bool = False) -> np.ndarray:
        o = np.ascontiguousarray(o, np.float64).reshape(-1, 3)
        d = np.ascontiguousarray(d, np.float64).reshape(-1, 3)
        out = np.zeros(o.shape[0], np.uint8)
        self.lib.pv3d_oracle_rays(self.h, _ptr(o), _ptr(d), o.shape[0], t_min, int(brute), _ptr(out))
        return out.astype(bool)


def _gen_arrays(gen):
    """Flatten a generator (duck-typed: attributes of scenes.Generator)."""
    m = gen.origin.shape[0]
    mod_f = np.zeros((m, 10), np.float32)
    mod_f[:, 0:3] = gen.origin
    mod_f[:, 3:6] = gen.u
    mod_f[:, 6:9] = gen.v
    mod_f[:, 9] = gen.pitch
    mod_i = np.stack([gen.cells_u, gen.cells_v, gen.layout, gen.tracker, gen.string], 1).astype(np.int32)
    offs, nsub, subs = [], [], []
    o = 0
    for lay in gen.layouts:
        offs.append(o)
        nsub.append(lay.n_sub)
        subs.append(np.asarray(lay.cell_sub, np.int32))
        o += len(lay.cell_sub)
    lay_off = np.asarray(offs, np.int32)
    lay_nsub = np.asarray(nsub, np.int32)
    lay_sub = np.concatenate(subs).astype(np.int32) if subs else np.zeros(1, np.int32)
    pivots = np.ascontiguousarray(gen.pivots, np.float32).reshape(-1, 3)
    if pivots.shape[0] == 0:
        pivots = np.zeros((1, 3), np.float32)
    return (np.ascontiguousarray(mod_f), np.ascontiguousarray(mod_i), lay_off, lay_nsub, lay_sub,
            int(gen.pivots.shape[0]), pivots)


def module_pmpp(g, cell_sub, n_sub, i_ref=I_REF, v_cell=V_CELL, v_diode=V_DIODE) -> float:
    lib = _load()
    g = np.ascontiguousarray(g, np.float64)
    cs = np.ascontiguousarray(cell_sub, np.int32)
    return lib.pv3d_oracle_module_pmpp(g.shape[0], _ptr(g), _ptr(cs), int(n_sub), i_ref, v_cell, v_diode)


def evaluate(scene, gen, sun, poses, n: int, map_res: int, steps=None, modules=None,
             want_mask: bool = True, brute: bool = False, threads: int | None = None,
             oscene: OracleScene | None = None, i_ref=I_REF, v_cell=V_CELL, v_diode=V_DIODE) -> dict:
    """Evaluate the oracle; arguments are duck-typed scenes.* objects.

    Returns a dict with counts [S, C], bits/mbits [S, C] (n <= 8), power,
    power_unshaded, cos_inc [S, M_eval], delta [S], cell_beam_loss [C],
    energy, energy_unshaded [M_eval], and the step/module index arrays.
    """
    lib = _load()
    if oscene is None:
        oscene = OracleScene(scene.verts, scene.tris)
    mod_f, mod_i, lay_off, lay_nsub, lay_sub, n_trk, pivots = _gen_arrays(gen)
    n_steps = sun.xyz.shape[0]
    steps = np.arange(n_steps, dtype=np.int64) if steps is None else np.asarray(steps, np.int64)
    mods = (np.arange(mod_f.shape[0], dtype=np.int32) if modules is None
            else np.asarray(modules, np.int32))
    if steps.size and (steps.min() < 0 or steps.max() >= n_steps):
        raise IndexError("step out of range")
    if mods.size and (mods.min() < 0 or mods.max() >= mod_f.shape[0]):
        raise IndexError("module out of range")
    cells = mod_i[mods, 0].astype(np.int64) * mod_i[mods, 1]
    C_ = int(cells.sum())
    S, Me = steps.size, mods.size
    sunxyz = np.ascontiguousarray(sun.xyz, np.float64)
    dni = np.ascontiguousarray(sun.dni, np.float32)
    dhi = np.ascontiguousarray(sun.dhi, np.float32)
    dt = np.ascontiguousarray(sun.dt_h, np.float32)
    if poses is None or n_trk == 0:
        pz = np.zeros((n_steps, 1, 2), np.float32)
    else:
        pz = np.ascontiguousarray(poses, np.float32)
    out = dict(
        counts=np.zeros((S, C_), np.int32),
        bits=np.zeros((S, C_), np.uint64) if n <= 8 else None,
        mbits=np.zeros((S, C_), np.uint64) if (n <= 8 and want_mask) else None,
        power=np.zeros((S, Me)), power_unshaded=np.zeros((S, Me)), cos_inc=np.zeros((S, Me)),
        delta=np.zeros(S), cell_beam_loss=np.zeros(C_), energy=np.zeros(Me),
        energy_unshaded=np.zeros(Me),
    )
    if threads is None:
        threads = os.cpu_count() or 1

    def p(a):
        return None if a is None else _ptr(a)
    rc = lib.pv3d_oracle_evaluate(
        oscene.h, mod_f.shape[0], _ptr(mod_f), _ptr(mod_i), _ptr(lay_off), _ptr(lay_nsub),
        _ptr(lay_sub), n_trk, _ptr(pivots), _ptr(sunxyz), _ptr(dni), _ptr(dhi), _ptr(dt), _ptr(pz),
        int(n), int(map_res), i_ref, v_cell, v_diode, _ptr(steps), S, _ptr(mods), Me,
        int(want_mask), int(brute), int(threads),
        _ptr(out["counts"]), p(out["bits"]), p(out["mbits"]), _ptr(out["power"]),
        _ptr(out["power_unshaded"]), _ptr(out["cos_inc"]), _ptr(out["delta"]),
        _ptr(out["cell_beam_loss"]), _ptr(out["energy"]), _ptr(out["energy_unshaded"]))
    if rc != 0:
        raise ValueError("oracle rejected its input")
    out["steps"] = steps
    out["modules"] = mods
    out["cells_per_module"] = cells
    return out


def evaluate_workload(w, **kw) -> dict:
    return evaluate(w.scene, w.gen, w.sun, w.poses, w.n, w.map_res, **kw)


def cell_beam_loss_from_counts(w, steps, modules, counts, cos_inc) -> np.ndarray:
    """Per-cell beam irradiation removed by shading (Section 2 step 4: the
    beam component is taken from the shaded share of a cell, then summed over
    time): sum over ``steps`` of DNI * max(0, cos_inc) * (count / n^2) * dt, in
    Wh/m^2, for given shaded-sample counts [S, C_eval] (cells of ``modules``
    in order) and the oracle's cosines of incidence [S, M_eval].  Used to
    bound results whose counts differ from the oracle's at masked samples."""
    gen, sun = w.gen, w.sun
    steps = np.asarray(steps, np.int64)
    mods = np.asarray(modules, np.int64)
    cells = (gen.cells_u[mods].astype(np.int64) * gen.cells_v[mods])
    mod_of_cell = np.repeat(np.arange(mods.size), cells)
    beam = sun.dni[steps].astype(np.float64)[:, None] * np.maximum(0.0, np.asarray(cos_inc, np.float64))
    beam = np.where(sun.xyz[steps, 2][:, None] > 0.0, beam, 0.0)
    f = np.asarray(counts, np.float64) / float(w.n * w.n)
    return (beam[:, mod_of_cell] * f * sun.dt_h[steps].astype(np.float64)[:, None]).sum(0)


def samples(gen, poses, step: int, module: int, n: int) -> np.ndarray:
    lib = _load()
    mod_f, mod_i, _, _, _, n_trk, pivots = _gen_arrays(gen)
    pz = (np.zeros((step + 1, 1, 2), np.float32) if poses is None or n_trk == 0
          else np.ascontiguousarray(poses, np.float32))
    nc = int(mod_i[module, 0]) * int(mod_i[module, 1])
    xyz = np.zeros((nc * n * n, 3))
    lib.pv3d_oracle_samples(mod_f.shape[0], _ptr(mod_f), _ptr(mod_i), n_trk, _ptr(pivots), _ptr(pz),
                            step, module, n, _ptr(xyz))
    return xyz


def module_normal(gen, poses, step: int, module: int) -> np.ndarray:
    lib = _load()
    mod_f, mod_i, _, _, _, n_trk, pivots = _gen_arrays(gen)
    pz = (np.zeros((step + 1, 1, 2), np.float32) if poses is None or n_trk == 0
          else np.ascontiguousarray(poses, np.float32))
    out = np.zeros(3)
    lib.pv3d_oracle_module_normal(mod_f.shape[0], _ptr(mod_f), _ptr(mod_i), n_trk, _ptr(pivots),
                                  _ptr(pz), step, module, _ptr(out))
    return out


def power_from_counts(w, steps, modules, counts, i_ref=I_REF, v_cell=V_CELL, v_diode=V_DIODE) -> np.ndarray:
    """Oracle PV model (Section 2, step 4) on given per-cell shaded counts
    [S, C_eval]; returns power [S, M_eval]."""
    lib = _load()
    gen, sun = w.gen, w.sun
    mod_f, mod_i, lay_off, lay_nsub, lay_sub, n_trk, pivots = _gen_arrays(gen)
    steps = np.ascontiguousarray(steps, np.int64)
    mods = np.ascontiguousarray(modules, np.int32)
    cnt = np.ascontiguousarray(counts, np.int32)
    pz = (np.zeros((sun.xyz.shape[0], 1, 2), np.float32) if w.poses is None or n_trk == 0
          else np.ascontiguousarray(w.poses, np.float32))
    out = np.zeros((steps.size, mods.size))
    lib.pv3d_oracle_power_from_counts(
        mod_f.shape[0], _ptr(mod_f), _ptr(mod_i), _ptr(lay_off), _ptr(lay_nsub), _ptr(lay_sub), n_trk,
        _ptr(pivots), _ptr(np.ascontiguousarray(sun.xyz, np.float64)), _ptr(np.ascontiguousarray(sun.dni, np.float32)),
        _ptr(np.ascontiguousarray(sun.dhi, np.float32)), _ptr(pz), int(w.n), i_ref, v_cell, v_diode,
        _ptr(steps), steps.size, _ptr(mods), mods.size, _ptr(cnt), _ptr(out))
    return out


def series_pmpp(ik, vk, v_diode=V_DIODE) -> float:
    """Maximum power of substrings (current limits ik, voltages vk) in one series string."""
    lib = _load()
    ik = np.ascontiguousarray(ik, np.float64)
    vk = np.ascontiguousarray(vk, np.float64)
    return lib.pv3d_oracle_series_pmpp(ik.size, _ptr(ik), _ptr(vk), v_diode)


def parallel_pmpp(strings, v_diode=V_DIODE) -> float:
    """Maximum power of series strings in parallel at one voltage; `strings`
    is a list of (ik, vk) substring current limits and voltages."""
    lib = _load()
    off = np.concatenate([[0], np.cumsum([len(a) for a, _ in strings])]).astype(np.int32)
    ik = np.ascontiguousarray(np.concatenate([a for a, _ in strings]), np.float64)
    vk = np.ascontiguousarray(np.concatenate([b for _, b in strings]), np.float64)
    return lib.pv3d_oracle_parallel_pmpp(len(strings), _ptr(off), _ptr(ik), _ptr(vk), v_diode)


def string_index(gen):
    """(strings, mod_string): the distinct string ids in ascending order, and
    each module's index into them."""
    ids, inv = np.unique(np.asarray(gen.string), return_inverse=True)
    return ids, inv.astype(np.int32)


def string_power_from_counts(w, steps, counts, i_ref=I_REF, v_cell=V_CELL, v_diode=V_DIODE):
    """Oracle string model (modules in series strings, one MPP per string) on
    given per-cell shaded counts [S, C] of every module; returns (power,
    power_unshaded) [S, n_strings], strings in ascending id order."""
    lib = _load()
    gen, sun = w.gen, w.sun
    mod_f, mod_i, lay_off, lay_nsub, lay_sub, n_trk, pivots = _gen_arrays(gen)
    ids, ms = string_index(gen)
    steps = np.ascontiguousarray(steps, np.int64)
    cnt = np.ascontiguousarray(counts, np.int32)
    pz = (np.zeros((sun.xyz.shape[0], 1, 2), np.float32) if w.poses is None or n_trk == 0
          else np.ascontiguousarray(w.poses, np.float32))
    p = np.zeros((steps.size, ids.size))
    pu = np.zeros((steps.size, ids.size))
    lib.pv3d_oracle_string_power_from_counts(
        mod_f.shape[0], _ptr(mod_f), _ptr(mod_i), _ptr(lay_off), _ptr(lay_nsub), _ptr(lay_sub), n_trk,
        _ptr(pivots), _ptr(np.ascontiguousarray(sun.xyz, np.float64)), _ptr(np.ascontiguousarray(sun.dni, np.float32)),
        _ptr(np.ascontiguousarray(sun.dhi, np.float32)), _ptr(pz), int(w.n), i_ref, v_cell, v_diode,
        _ptr(steps), steps.size, _ptr(ms), ids.size, _ptr(cnt), _ptr(p), _ptr(pu), None, 0, None, None)
    return p, pu


def array_index(gen):
    """(arrays, str_array): the distinct array ids of the generator's modules in
    ascending order, and each string's index into them (the strings in
    ascending string id; all modules of a string share one array id)."""
    arr = np.zeros(len(gen.string), np.int32) if getattr(gen, "array", None) is None else np.asarray(gen.array)
    sid, ms = string_index(gen)
    a_ids = np.unique(arr)
    str_array = np.zeros(sid.size, np.int32)
    str_array[ms] = np.searchsorted(a_ids, arr)
    return a_ids, str_array


def array_power_from_counts(w, steps, counts, i_ref=I_REF, v_cell=V_CELL, v_diode=V_DIODE):
    """Oracle model of the arrays of strings in parallel (one voltage and one
    maximum power point per array) on given per-cell shaded counts [S, C];
    returns (power, power_unshaded) [S, n_arrays], arrays in ascending id."""
    lib = _load()
    gen, sun = w.gen, w.sun
    mod_f, mod_i, lay_off, lay_nsub, lay_sub, n_trk, pivots = _gen_arrays(gen)
    ids, ms = string_index(gen)
    a_ids, str_array = array_index(gen)
    steps = np.ascontiguousarray(steps, np.int64)
    cnt = np.ascontiguousarray(counts, np.int32)
    pz = (np.zeros((sun.xyz.shape[0], 1, 2), np.float32) if w.poses is None or n_trk == 0
          else np.ascontiguousarray(w.poses, np.float32))
    p = np.zeros((steps.size, ids.size)); pu = np.zeros((steps.size, ids.size))
    ap = np.zeros((steps.size, a_ids.size)); apu = np.zeros((steps.size, a_ids.size))
    lib.pv3d_oracle_string_power_from_counts(
        mod_f.shape[0], _ptr(mod_f), _ptr(mod_i), _ptr(lay_off), _ptr(lay_nsub), _ptr(lay_sub), n_trk,
        _ptr(pivots), _ptr(np.ascontiguousarray(sun.xyz, np.float64)), _ptr(np.ascontiguousarray(sun.dni, np.float32)),
        _ptr(np.ascontiguousarray(sun.dhi, np.float32)), _ptr(pz), int(w.n), i_ref, v_cell, v_diode,
        _ptr(steps), steps.size, _ptr(ms), ids.size, _ptr(cnt), _ptr(p), _ptr(pu), _ptr(str_array), a_ids.size,
        _ptr(ap), _ptr(apu))
    return ap, apu


def sun_table(lat_deg: float, day_first: int, n_days: int, step_h: float, daylight_only: bool = True,
              dhi_fraction: float = 0.1):
    """Clear-sky sun table (see pv3d_oracle_sun_table): (xyz [N, 3], dni [N], dhi [N])."""
    lib = _load()
    n = lib.pv3d_oracle_sun_table(lat_deg, day_first, n_days, step_h, int(daylight_only), dhi_fraction,
                                  None, None, None)
    xyz = np.zeros((n, 3)); dni = np.zeros(n); dhi = np.zeros(n)
    lib.pv3d_oracle_sun_table(lat_deg, day_first, n_days, step_h, int(daylight_only), dhi_fraction,
                              _ptr(xyz), _ptr(dni), _ptr(dhi))
    return xyz, dni, dhi


def heat_map(sun_xyz, p_gen, pu_gen, dt_h, n_az: int, n_zen: int):
    """Effective-shading map of the generator over the sky (the paper's Fig. 6:
    the shading factor as a function of the sun's azimuth and zenith): the
    steps with the sun above the horizon are binned by compass azimuth
    [0, 360) in n_az bins and zenith [0, 90] in n_zen bins (the last bin
    closed); per bin the sums of the generator's energy sum_steps P * dt with
    and without shading and the step count.  The bin's effective shading factor
    is 1 - E / E_unshaded."""
    s = np.asarray(sun_xyz, np.float64)
    up = s[:, 2]
    lit = up > 0
    az = np.degrees(np.arctan2(s[:, 0], s[:, 1])) % 360.0
    zen = np.degrees(np.arccos(np.clip(up, -1.0, 1.0)))
    ia = np.minimum((az / 360.0 * n_az).astype(np.int64), n_az - 1)
    iz = np.minimum((zen / 90.0 * n_zen).astype(np.int64), n_zen - 1)
    e = np.zeros((n_zen, n_az)); eu = np.zeros((n_zen, n_az)); cnt = np.zeros((n_zen, n_az), np.int64)
    dt = np.asarray(dt_h, np.float64)
    np.add.at(e, (iz[lit], ia[lit]), (np.asarray(p_gen, np.float64) * dt)[lit])
    np.add.at(eu, (iz[lit], ia[lit]), (np.asarray(pu_gen, np.float64) * dt)[lit])
    np.add.at(cnt, (iz[lit], ia[lit]), 1)
    return e, eu, cnt


def sky_patches(rings: int, sectors: int):
    """Sky directions for diffuse shading (reading of the isotropic diffuse
    term of Section 2, step 4, which the paper leaves unshaded): the upper
    hemisphere cut into `rings` zenith bands of equal angle over [0, 90] deg
    and `sectors` equal azimuth sectors; each patch is represented by the
    direction at its centre angles and carries its solid angle
    (cos z0 - cos z1) * 2 pi / sectors.  Returns (xyz [rings*sectors, 3],
    solid angle [rings*sectors]), ring-major, azimuth clockwise from north."""
    out, dom = [], []
    for r in range(rings):
        z0, z1 = math.pi / 2 * r / rings, math.pi / 2 * (r + 1) / rings
        zc = 0.5 * (z0 + z1)
        for k in range(sectors):
            a = 2 * math.pi * (k + 0.5) / sectors
            out.append((math.sin(zc) * math.sin(a), math.sin(zc) * math.cos(a), math.cos(zc)))
            dom.append((math.cos(z0) - math.cos(z1)) * 2 * math.pi / sectors)
    return np.array(out), np.array(dom)


def diffuse_shade_fractions(w, rings: int, sectors: int, counts, normals):
    """Per cell, the share of the isotropic diffuse irradiance it loses to
    obstructions: the sky patches weighted by solid angle times the cosine to
    the module's front normal (where positive), and the fraction of the cell's
    samples shaded toward each patch (counts [patch, cell] out of n^2):
    f = sum_p W_p s_p / sum_p W_p.  `normals` [cells, 3] are the cells'
    module normals.  Unobstructed, f = 0."""
    xyz, dom = sky_patches(rings, sectors)
    wgt = dom[:, None] * np.maximum(0.0, xyz @ np.asarray(normals, np.float64).T)   # [patch, cell]
    frac = np.asarray(counts, np.float64) / float(w.n * w.n)
    tot = wgt.sum(0)
    return np.where(tot > 0, (wgt * frac).sum(0) / np.where(tot > 0, tot, 1.0), 0.0)


def pose_bins(az_tilt, n_az: int, n_tilt: int):
    """Pose bins of tracker poses for the diffuse shading of tracked modules
    (reading: a tracker's view of the sky changes with its pose, Section 3.4;
    the sky view is taken once per bin): compass azimuth in ``n_az`` equal
    sectors of [0, 2 pi), tilt in ``n_tilt`` equal bands of [0, pi/2], bin =
    band * n_az + sector.  ``az_tilt`` [S, 2] (radians).  Returns (bin [S],
    centre azimuth [n_az * n_tilt], centre tilt [n_az * n_tilt]), the centre
    being the middle of both ranges."""
    a = np.asarray(az_tilt, np.float64).reshape(-1, 2)
    two_pi, half_pi = 2.0 * math.pi, 0.5 * math.pi
    az = np.mod(a[:, 0], two_pi)
    ia = np.clip(np.floor(az / two_pi * n_az).astype(np.int64), 0, n_az - 1)
    it = np.clip(np.floor(np.clip(a[:, 1], 0.0, half_pi) / half_pi * n_tilt).astype(np.int64), 0, n_tilt - 1)
    b = np.arange(n_az * n_tilt)
    return it * n_az + ia, (b % n_az + 0.5) * two_pi / n_az, (b // n_az + 0.5) * half_pi / n_tilt


def tracked_diffuse_fractions(w, rings: int, sectors: int, n_az: int, n_tilt: int, n: int, map_res: int,
                              bins=None, want_mask: bool = True):
    """Diffuse shading fractions of a tracked generator per pose bin: a
    step's bin is that of the first tracker's pose (pose_bins); for each bin
    (those of the lit steps, or ``bins``) every tracker takes the bin's
    centre pose and the exact rays toward the sky patches give each cell's
    fraction (diffuse_shade_fractions, with the module normals at that pose).
    Returns ({bin: fractions [C]}, {bin: masked share [C]} (the patches'
    masked samples weighted like the fraction, or None), the step bins [S])."""
    gen = w.gen
    step_bin, az_c, tilt_c = pose_bins(w.poses[:, 0, :], n_az, n_tilt)
    lit = w.sun.xyz[:, 2] > 0
    use = sorted(set(int(b) for b in step_bin[lit])) if bins is None else list(bins)
    xyz, dom = sky_patches(rings, sectors)
    P = len(xyz)
    sun = type(w.sun)(xyz=xyz, dni=np.ones(P, np.float32), dhi=np.zeros(P, np.float32), dt_h=np.ones(P, np.float32))
    n_trk = gen.pivots.shape[0]
    cells = (gen.cells_u.astype(np.int64) * gen.cells_v)
    out, masked = {}, {}
    for b in use:
        poses = np.zeros((P, n_trk, 2), np.float32)
        poses[:, :, 0] = az_c[b]
        poses[:, :, 1] = tilt_c[b]
        o = evaluate(w.scene, gen, sun, poses, n, map_res, want_mask=want_mask)
        normals = np.concatenate([np.repeat(module_normal(gen, poses, 0, m)[None, :], cells[m], 0)
                                  for m in range(gen.n_modules)])
        wn = type(w)(w.name, w.scene, gen, sun, poses, n, map_res)
        out[b] = diffuse_shade_fractions(wn, rings, sectors, o["counts"], normals)
        if want_mask:
            wgt = dom[:, None] * np.maximum(0.0, xyz @ normals.T)
            mk = popcount64(o["mbits"]) / float(n * n)
            masked[b] = (wgt * mk).sum(0) / np.maximum(wgt.sum(0), 1e-300)
        else:
            masked[b] = None
    return out, masked, step_bin


def popcount64(a: np.ndarray) -> np.ndarray:
    a = a.astype(np.uint64)
    c = np.zeros(a.shape, np.int32)
    for k in range(64):
        c += ((a >> np.uint64(k)) & np.uint64(1)).astype(np.int32)
    return c


def unpack_bits(bits: np.ndarray, n: int) -> np.ndarray:
    """[..., cells] uint64 -> [..., cells, n*n] bool (sample k = j*n + i)."""
    k = np.arange(n * n, dtype=np.uint64)
    return ((bits[..., None] >> k) & np.uint64(1)).astype(bool)
