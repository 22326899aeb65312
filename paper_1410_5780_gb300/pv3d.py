"""Thin Python binding of the pv3d C ABI (include/pv3d.h).

Argument marshalling only: every step of the shadow-sample path runs in the
CUDA library.  The functions keep the C names (pv3d_create, pv3d_scene_load,
...); ``Context`` wraps a handle and turns numpy inputs into the C structs.
Device outputs are torch tensors (PyTorch provides device memory and the
stream); host outputs are numpy arrays.  There is no fallback: if the library
is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

PV3D_OK = 0
PV3D_E_INVALID = -1
PV3D_E_NOMEM = -2
PV3D_E_ADMISSION = -3
PV3D_E_OVERFLOW = -4
PV3D_E_TIMEOUT = -5
PV3D_E_DEVICE = -6
PV3D_E_PENDING = -7
PV3D_E_NOTFOUND = -8
PV3D_E_TOOBIG = -9
PV3D_NOALLOC_MAX_RES = 2048
PV3D_DEPTH_F32 = 0
PV3D_DEPTH_U24 = 1
PV3D_PATH_FUSED = 0
PV3D_PATH_MAP = 1
PV3D_WINDOWS_ONE = 0
PV3D_WINDOWS_PER_TRACKER = 1
PV3D_WINDOWS_PER_STRING = 2
PV3D_WINDOWS_PER_ARRAY = 3

EXPORTED = ("pv3d_create", "pv3d_destroy", "pv3d_last_error", "pv3d_scene_load", "pv3d_generator_define",
            "pv3d_set_poses", "pv3d_set_sun", "pv3d_evaluate", "pv3d_submit", "pv3d_poll", "pv3d_release",
            "pv3d_last_profile", "pv3d_module_shade_noalloc", "pv3d_evaluate_batch", "pv3d_generator_strings",
            "pv3d_set_sun_clear_sky", "pv3d_sun_table", "pv3d_sky_view", "pv3d_generator_arrays",
            "pv3d_raster_peak")


class pv3d_opts(C.Structure):
    _fields_ = [("device", C.c_int32), ("map_res", C.c_int32), ("tile", C.c_int32), ("chunk_steps", C.c_int32),
                ("depth_format", C.c_int32), ("max_inflight", C.c_int32), ("hbm_budget_bytes", C.c_int64),
                ("wave_scratch_mb", C.c_int32), ("reserved0", C.c_int32), ("bin_capacity", C.c_int64),
                ("reserved", C.c_int32 * 4)]


class pv3d_module(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("u", C.c_float * 3), ("v", C.c_float * 3), ("pitch", C.c_float),
                ("cells_u", C.c_int32), ("cells_v", C.c_int32), ("layout", C.c_int32), ("tracker", C.c_int32),
                ("string_id", C.c_int32), ("array_id", C.c_int32)]


class pv3d_layout(C.Structure):
    _fields_ = [("cells_u", C.c_int32), ("cells_v", C.c_int32), ("n_sub", C.c_int32), ("reserved", C.c_int32),
                ("cell_sub", C.POINTER(C.c_int32))]


class pv3d_tracker(C.Structure):
    _fields_ = [("pivot", C.c_float * 3)]


class pv3d_eval_opts(C.Structure):
    _fields_ = [("samples_per_side", C.c_int32), ("map_res", C.c_int32), ("step_begin", C.c_int64),
                ("step_end", C.c_int64), ("i_ref", C.c_float), ("v_cell", C.c_float), ("v_diode", C.c_float),
                ("chunk_steps", C.c_int32), ("stream", C.c_void_p), ("path", C.c_int32),
                ("profile", C.c_int32), ("diffuse_shading", C.c_int32), ("window_groups", C.c_int32),
                ("reserved", C.c_int32 * 4)]


class pv3d_profile(C.Structure):
    _fields_ = [("n_stages", C.c_int32), ("waves", C.c_int32), ("stage_ms", C.c_float * 8),
                ("device_ms", C.c_float), ("reserved0", C.c_int32), ("sample_tests", C.c_int64),
                ("texel_visits", C.c_int64), ("texel_writes", C.c_int64), ("tris_culled", C.c_int64),
                ("nonempty_tiles", C.c_int64), ("binned_tris", C.c_int64), ("candidates", C.c_int64),
                ("dense_tiles", C.c_int64), ("sample_tiles", C.c_int64), ("pair_tests", C.c_int64),
                ("heavy_tiles", C.c_int64), ("heavy_sample_tests", C.c_int64), ("heavy_texel_writes", C.c_int64),
                ("heavy_why", C.c_int64 * 3)]


STAGES = ("setup", "bin", "raster", "heavy", "pv", "epilogue")


class pv3d_result(C.Structure):
    _fields_ = [("is_device", C.c_int32), ("reserved0", C.c_int32),
                ("energy", C.c_void_p), ("energy_unshaded", C.c_void_p), ("power", C.c_void_p),
                ("power_unshaded", C.c_void_p), ("cell_beam_loss", C.c_void_p), ("cell_counts", C.c_void_p),
                ("sample_bits", C.c_void_p), ("tests", C.c_int64), ("steps_lit", C.c_int64),
                ("device_ms", C.c_float), ("waves", C.c_int32), ("nonempty_tiles", C.c_int64),
                ("binned_tris", C.c_int64), ("kernel_launches", C.c_int64), ("latency_ms", C.c_float),
                ("reserved1", C.c_int32), ("string_energy", C.c_void_p), ("string_energy_unshaded", C.c_void_p),
                ("string_power", C.c_void_p), ("string_power_unshaded", C.c_void_p),
                ("heat_az_bins", C.c_int32), ("heat_zen_bins", C.c_int32), ("heat_energy", C.c_void_p),
                ("heat_energy_unshaded", C.c_void_p), ("heat_steps", C.c_void_p),
                ("array_energy", C.c_void_p), ("array_energy_unshaded", C.c_void_p), ("array_power", C.c_void_p),
                ("array_power_unshaded", C.c_void_p)]


class pv3d_sky_view_opts(C.Structure):
    _fields_ = [("rings", C.c_int32), ("sectors", C.c_int32), ("samples_per_side", C.c_int32),
                ("map_res", C.c_int32), ("pose_az_bins", C.c_int32), ("pose_tilt_bins", C.c_int32),
                ("reserved", C.c_int32 * 2)]


class pv3d_sky_opts(C.Structure):
    _fields_ = [("latitude_deg", C.c_double), ("step_h", C.c_double), ("day_first", C.c_int32),
                ("n_days", C.c_int32), ("daylight_only", C.c_int32), ("dhi_fraction", C.c_float),
                ("tracker_tilt_max_deg", C.c_float), ("reserved", C.c_int32 * 5)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libpv3d.so; raise if it is not built (no CPU fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"pv3d CUDA library not built ({path}); run paper_1410_5780_gb300.build.build()")
            _build.build()
        lib = C.CDLL(path)
        P = C.c_void_p
        lib.pv3d_create.argtypes = [C.POINTER(P), C.POINTER(pv3d_opts)]
        lib.pv3d_destroy.argtypes = [P]
        lib.pv3d_destroy.restype = None
        lib.pv3d_last_error.argtypes = [P]
        lib.pv3d_last_error.restype = C.c_char_p
        lib.pv3d_scene_load.argtypes = [P, P, C.c_int64, P, C.c_int64, C.POINTER(C.c_uint32)]
        lib.pv3d_generator_define.argtypes = [P, C.c_uint32, C.POINTER(pv3d_module), C.c_int32,
                                              C.POINTER(pv3d_layout), C.c_int32, C.POINTER(pv3d_tracker), C.c_int32,
                                              C.POINTER(C.c_uint32)]
        lib.pv3d_set_poses.argtypes = [P, C.c_uint32, P, C.c_int64]
        lib.pv3d_set_sun.argtypes = [P, C.c_uint32, P, P, P, P, C.c_int64]
        lib.pv3d_evaluate.argtypes = [P, C.c_uint32, C.POINTER(pv3d_eval_opts), C.POINTER(pv3d_result)]
        lib.pv3d_submit.argtypes = [P, C.c_uint32, C.POINTER(pv3d_eval_opts), C.POINTER(pv3d_result),
                                    C.POINTER(C.c_uint64)]
        lib.pv3d_poll.argtypes = [P, C.c_uint64, C.c_int32]
        lib.pv3d_release.argtypes = [P, C.c_uint32]
        lib.pv3d_last_profile.argtypes = [P, C.POINTER(pv3d_profile)]
        lib.pv3d_generator_strings.argtypes = [P, C.c_uint32, C.POINTER(C.c_int32), P]
        lib.pv3d_generator_arrays.argtypes = [P, C.c_uint32, C.POINTER(C.c_int32), P]
        lib.pv3d_set_sun_clear_sky.argtypes = [P, C.c_uint32, C.POINTER(pv3d_sky_opts), C.POINTER(C.c_int64)]
        lib.pv3d_sun_table.argtypes = [P, C.c_uint32, P, P, P, P, C.c_int64]
        lib.pv3d_sky_view.argtypes = [P, C.c_uint32, C.POINTER(pv3d_sky_view_opts), P]
        lib.pv3d_evaluate_batch.argtypes = [P, C.c_int32, P, C.POINTER(pv3d_eval_opts), C.POINTER(pv3d_result)]
        lib.pv3d_module_shade_noalloc.argtypes = [P, C.c_int64, C.POINTER(pv3d_module), P, C.c_int32, C.c_int32,
                                                  P, P]
        lib.pv3d_raster_peak.argtypes = [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        for name in EXPORTED:
            if name not in ("pv3d_destroy", "pv3d_last_error"):
                getattr(lib, name).restype = C.c_int
        _lib = lib
        return lib


class PV3DError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pv3d error {code}: {msg}")
        self.code = code


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


OUTPUTS = ("energy", "energy_unshaded", "power", "power_unshaded", "cell_beam_loss", "cell_counts", "sample_bits")


class Context:
    """One pv3d context (one device, one host thread)."""

    def __init__(self, device: int = 0, map_res: int = 0, tile: int = 0, chunk_steps: int = 0,
                 depth_format: int = PV3D_DEPTH_F32, max_inflight: int = 0, hbm_budget_bytes: int = 0,
                 wave_scratch_mb: int = 0, bin_capacity: int = 0):
        self.lib = load()
        o = pv3d_opts(device=device, map_res=map_res, tile=tile, chunk_steps=chunk_steps,
                      depth_format=depth_format, max_inflight=max_inflight, hbm_budget_bytes=hbm_budget_bytes,
                      wave_scratch_mb=wave_scratch_mb, bin_capacity=bin_capacity)
        h = C.c_void_p()
        rc = self.lib.pv3d_create(C.byref(h), C.byref(o))
        if rc != 0:
            raise PV3DError(rc, "pv3d_create failed")
        self.h = h
        self.device = device
        self._gens = {}
        self._keep = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.pv3d_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc):
        if rc != 0 and rc != PV3D_E_PENDING:
            raise PV3DError(rc, self.lib.pv3d_last_error(self.h).decode())
        return rc

    # ---- step 1 ------------------------------------------------------------
    def scene_load(self, verts: np.ndarray, tris: np.ndarray) -> int:
        v = np.ascontiguousarray(verts, np.float32).reshape(-1, 3)
        t = np.ascontiguousarray(tris, np.int32).reshape(-1, 3)
        sid = C.c_uint32()
        self._check(self.lib.pv3d_scene_load(self.h, _p(v), v.shape[0], _p(t), t.shape[0], C.byref(sid)))
        return sid.value

    # ---- step 2 ------------------------------------------------------------
    def generator_define(self, scene_id: int, gen) -> int:
        """``gen`` carries origin, u, v, cells_u, cells_v, pitch, layout, tracker,
        string arrays, a ``layouts`` list (cells_u, cells_v, n_sub, cell_sub) and
        ``pivots`` (attributes of paper_1410_5780_gb300.scenes.Generator)."""
        m = int(gen.origin.shape[0])
        mods = (pv3d_module * m)()
        mv = np.ctypeslib.as_array(mods)  # a structured view of the same memory
        mv["origin"] = np.asarray(gen.origin, np.float32).reshape(m, 3)
        mv["u"] = np.asarray(gen.u, np.float32).reshape(m, 3)
        mv["v"] = np.asarray(gen.v, np.float32).reshape(m, 3)
        mv["pitch"] = np.asarray(gen.pitch, np.float32).reshape(m)
        mv["cells_u"] = np.asarray(gen.cells_u).reshape(m)
        mv["cells_v"] = np.asarray(gen.cells_v).reshape(m)
        mv["layout"] = np.asarray(gen.layout).reshape(m)
        mv["tracker"] = np.asarray(gen.tracker).reshape(m)
        mv["string_id"] = np.asarray(gen.string).reshape(m)
        mv["array_id"] = 0 if getattr(gen, "array", None) is None else np.asarray(gen.array).reshape(m)
        subs = [np.ascontiguousarray(l.cell_sub, np.int32) for l in gen.layouts]
        lays = (pv3d_layout * len(subs))()
        for i, (l, s) in enumerate(zip(gen.layouts, subs)):
            lays[i].cells_u = int(l.cells_u); lays[i].cells_v = int(l.cells_v); lays[i].n_sub = int(l.n_sub)
            lays[i].cell_sub = s.ctypes.data_as(C.POINTER(C.c_int32))
        piv = np.asarray(gen.pivots, np.float32).reshape(-1, 3)
        trk = (pv3d_tracker * max(1, piv.shape[0]))()
        if piv.shape[0]:
            np.ctypeslib.as_array(trk)["pivot"] = piv
        gid = C.c_uint32()
        self._check(self.lib.pv3d_generator_define(self.h, scene_id, mods, m, lays, len(subs), trk, piv.shape[0],
                                                   C.byref(gid)))
        cells = int((np.asarray(gen.cells_u, np.int64) * np.asarray(gen.cells_v, np.int64)).sum())
        self._gens[gid.value] = {"modules": m, "cells": cells, "steps": 0, "strings": len(self.string_ids(gid.value)),
                                 "arrays": len(self.array_ids(gid.value)), "trackers": int(piv.shape[0])}
        return gid.value

    def array_ids(self, gen_id: int) -> np.ndarray:
        """pv3d_generator_arrays: the generator's distinct array ids, ascending
        (the order of the array outputs)."""
        n = C.c_int32()
        self._check(self.lib.pv3d_generator_arrays(self.h, gen_id, C.byref(n), None))
        ids = np.zeros(n.value, np.int32)
        self._check(self.lib.pv3d_generator_arrays(self.h, gen_id, C.byref(n), _p(ids)))
        return ids

    def string_ids(self, gen_id: int) -> np.ndarray:
        """pv3d_generator_strings: the generator's distinct string ids, ascending
        (the order of the string outputs)."""
        n = C.c_int32()
        self._check(self.lib.pv3d_generator_strings(self.h, gen_id, C.byref(n), None))
        ids = np.zeros(n.value, np.int32)
        self._check(self.lib.pv3d_generator_strings(self.h, gen_id, C.byref(n), _p(ids)))
        return ids

    def set_poses(self, gen_id: int, az_tilt: np.ndarray):
        a = np.ascontiguousarray(az_tilt, np.float32)
        self._check(self.lib.pv3d_set_poses(self.h, gen_id, _p(a), a.shape[0]))

    def set_sun(self, gen_id: int, sun_xyz, dni, dhi, dt_h):
        s = np.ascontiguousarray(sun_xyz, np.float64).reshape(-1, 3)
        a = np.ascontiguousarray(dni, np.float32)
        b = np.ascontiguousarray(dhi, np.float32)
        d = np.ascontiguousarray(dt_h, np.float32)
        self._check(self.lib.pv3d_set_sun(self.h, gen_id, _p(s), _p(a), _p(b), _p(d), s.shape[0]))
        self._gens[gen_id]["steps"] = s.shape[0]

    def set_sun_clear_sky(self, gen_id: int, latitude_deg: float, step_h: float, day_first: int = 1,
                          n_days: int = 365, daylight_only: bool = True, dhi_fraction: float = 0.1,
                          tracker_tilt_max_deg: float = 0.0) -> int:
        """pv3d_set_sun_clear_sky: the sun table (and, with a tilt limit, ideal
        tracker poses) computed on the device.  Returns the number of steps."""
        o = pv3d_sky_opts(latitude_deg=latitude_deg, step_h=step_h, day_first=day_first, n_days=n_days,
                          daylight_only=int(daylight_only), dhi_fraction=dhi_fraction,
                          tracker_tilt_max_deg=tracker_tilt_max_deg)
        n = C.c_int64()
        self._check(self.lib.pv3d_set_sun_clear_sky(self.h, gen_id, C.byref(o), C.byref(n)))
        self._gens[gen_id]["steps"] = n.value
        return n.value

    def sky_view(self, gen_id: int, rings: int = 9, sectors: int = 36, n: int = 3, map_res: int = 0,
                 pose_az_bins: int = 12, pose_tilt_bins: int = 6) -> np.ndarray:
        """pv3d_sky_view: per-cell diffuse shading fractions (kept with the
        generator for evaluations with diffuse_shading): [cells] for a
        generator of fixed modules, [pose_tilt_bins * pose_az_bins, cells]
        (one row per pose bin) for a tracked one."""
        o = pv3d_sky_view_opts(rings=rings, sectors=sectors, samples_per_side=n, map_res=map_res,
                               pose_az_bins=pose_az_bins, pose_tilt_bins=pose_tilt_bins)
        g = self._gens.get(gen_id, {"cells": 0, "trackers": 0})
        bins = pose_az_bins * pose_tilt_bins if g["trackers"] else 1
        f = np.zeros((bins, max(g["cells"], 1)), np.float32)
        self._check(self.lib.pv3d_sky_view(self.h, gen_id, C.byref(o), _p(f)))
        return f if g["trackers"] else f[0]

    def sun_table(self, gen_id: int):
        """pv3d_sun_table: (xyz [N, 3] float64, dni, dhi, dt_h [N] float32) of the generator."""
        n = self._gens[gen_id]["steps"]
        xyz = np.zeros((n, 3)); dni = np.zeros(n, np.float32); dhi = np.zeros(n, np.float32)
        dt = np.zeros(n, np.float32)
        self._check(self.lib.pv3d_sun_table(self.h, gen_id, _p(xyz), _p(dni), _p(dhi), _p(dt), n))
        return xyz, dni, dhi, dt

    # ---- steps 3 and 4 -----------------------------------------------------
    def _opts(self, n, map_res, step_begin, step_end, chunk_steps, stream, i_ref, v_cell, v_diode, path=0,
              profile=0, diffuse=False, window_groups=0):
        return pv3d_eval_opts(samples_per_side=n, map_res=map_res, step_begin=step_begin, step_end=step_end,
                              chunk_steps=chunk_steps, stream=stream, i_ref=i_ref, v_cell=v_cell, v_diode=v_diode,
                              path=path, profile=profile, diffuse_shading=int(diffuse),
                              window_groups=int(window_groups))

    def _alloc(self, gen_id, step_begin, step_end, outputs, device, heat_bins=None):
        if gen_id not in self._gens:  # let the library report the unknown id
            return pv3d_result(is_device=1 if device else 0), {}
        g = self._gens[gen_id]
        m, cells, n_steps, ns, na = g["modules"], g["cells"], g["steps"], g["strings"], g["arrays"]
        S = (step_end or n_steps) - step_begin
        shapes = dict(energy=((m,), "f8"), energy_unshaded=((m,), "f8"), power=((S, m), "f4"),
                      power_unshaded=((S, m), "f4"), cell_beam_loss=((cells,), "f8"),
                      cell_counts=((S, cells), "u1"), sample_bits=((S, cells), "u8"),
                      string_energy=((ns,), "f8"), string_energy_unshaded=((ns,), "f8"),
                      string_power=((S, ns), "f4"), string_power_unshaded=((S, ns), "f4"),
                      array_energy=((na,), "f8"), array_energy_unshaded=((na,), "f8"),
                      array_power=((S, na), "f4"), array_power_unshaded=((S, na), "f4"))
        if heat_bins:
            n_az, n_zen = heat_bins
            shapes.update(heat_energy=((n_zen, n_az), "f8"), heat_energy_unshaded=((n_zen, n_az), "f8"),
                          heat_steps=((n_zen, n_az), "i4"))
            outputs = tuple(outputs) + tuple(k for k in ("heat_energy", "heat_energy_unshaded", "heat_steps")
                                             if k not in outputs)
        res = pv3d_result(is_device=1 if device else 0)
        if heat_bins:
            res.heat_az_bins, res.heat_zen_bins = int(heat_bins[0]), int(heat_bins[1])
        arrays = {}
        for name in outputs:
            shape, dt = shapes[name]
            if device:
                import torch
                tdt = {"f8": torch.float64, "f4": torch.float32, "u1": torch.uint8, "u8": torch.int64,
                       "i4": torch.int32}[dt]
                a = torch.empty(shape, dtype=tdt, device=f"cuda:{self.device}")
                setattr(res, name, a.data_ptr())
            else:
                a = np.zeros(shape, dt)
                setattr(res, name, a.ctypes.data)
            arrays[name] = a
        return res, arrays

    def evaluate(self, gen_id: int, n: int = 3, map_res: int = 0, step_begin: int = 0, step_end: int = 0,
                 chunk_steps: int = 0, outputs=("energy", "energy_unshaded"), device: bool = True,
                 stream=None, i_ref: float = 0.0, v_cell: float = 0.0, v_diode: float = 0.0,
                 path: int = PV3D_PATH_FUSED, profile: bool = False, heat_bins=None,
                 diffuse_shading: bool = False, window_groups: int = PV3D_WINDOWS_ONE) -> dict:
        """pv3d_evaluate.  Returns the requested outputs (torch tensors on the
        device if ``device`` else numpy arrays) plus the counters.  ``heat_bins``
        = (azimuth bins, zenith bins) adds the sky map of the effective shading;
        ``window_groups`` (PV3D_WINDOWS_*) gives each tracker, string or array
        its own light window of side ``map_res``."""
        if stream is None and device:
            import torch
            stream = torch.cuda.current_stream(self.device).cuda_stream
        res, arrays = self._alloc(gen_id, step_begin, step_end, outputs, device, heat_bins)
        o = self._opts(n, map_res, step_begin, step_end, chunk_steps, stream, i_ref, v_cell, v_diode, path,
                       int(profile), diffuse_shading, window_groups)
        self._check(self.lib.pv3d_evaluate(self.h, gen_id, C.byref(o), C.byref(res)))
        arrays.update(tests=res.tests, steps_lit=res.steps_lit, device_ms=res.device_ms, waves=res.waves,
                      nonempty_tiles=res.nonempty_tiles, binned_tris=res.binned_tris,
                      kernel_launches=res.kernel_launches)
        return arrays

    def last_profile(self) -> dict:
        """pv3d_last_profile as a dict (stage times in ms, work counters)."""
        p = pv3d_profile()
        self._check(self.lib.pv3d_last_profile(self.h, C.byref(p)))
        d = {f"{name}_ms": p.stage_ms[k] for k, name in enumerate(STAGES)}
        d.update(waves=p.waves, device_ms=p.device_ms, sample_tests=p.sample_tests, texel_visits=p.texel_visits,
                 texel_writes=p.texel_writes, tris_culled=p.tris_culled, nonempty_tiles=p.nonempty_tiles,
                 binned_tris=p.binned_tris, candidates=p.candidates, dense_tiles=p.dense_tiles,
                 sample_tiles=p.sample_tiles, pair_tests=p.pair_tests, heavy_tiles=p.heavy_tiles,
                 heavy_sample_tests=p.heavy_sample_tests, heavy_texel_writes=p.heavy_texel_writes,
                 heavy_why=list(p.heavy_why))
        return d

    def submit(self, gen_id: int, n: int = 3, map_res: int = 0, step_begin: int = 0, step_end: int = 0,
               chunk_steps: int = 0, outputs=("energy", "energy_unshaded"), device: bool = True,
               stream=None, diffuse_shading: bool = False):
        """pv3d_submit.  Returns (request id, outputs dict); the outputs are
        valid once pv3d_poll returns PV3D_OK for the request (string and array
        outputs included; sky-map outputs and window groups are pv3d_evaluate's
        only)."""
        res, arrays = self._alloc(gen_id, step_begin, step_end, outputs, device)
        o = self._opts(n, map_res, step_begin, step_end, chunk_steps, None, 0.0, 0.0, 0.0,
                       diffuse=diffuse_shading)
        rid = C.c_uint64()
        self._check(self.lib.pv3d_submit(self.h, gen_id, C.byref(o), C.byref(res), C.byref(rid)))
        self._keep[rid.value] = (res, o, arrays)
        return rid.value, arrays

    def poll(self, req: int, timeout_ms: int = 0) -> int:
        rc = self.lib.pv3d_poll(self.h, req, timeout_ms)
        self._check(rc)
        if rc == PV3D_OK:
            res, _, arrays = self._keep.pop(req)
            arrays.update(tests=res.tests, steps_lit=res.steps_lit, device_ms=res.device_ms, waves=res.waves,
                          latency_ms=res.latency_ms)
        elif rc != PV3D_E_PENDING:
            self._keep.pop(req, None)
        return rc

    def evaluate_batch(self, gen_ids, n=3, map_res=0, chunk_steps=0, outputs=("energy", "energy_unshaded"),
                       device: bool = True) -> list:
        """pv3d_evaluate_batch over ``gen_ids``; ``n`` and ``map_res`` may be
        per-generator sequences."""
        k = len(gen_ids)
        ns = list(n) if hasattr(n, "__len__") else [n] * k
        rs = list(map_res) if hasattr(map_res, "__len__") else [map_res] * k
        ids = (C.c_uint32 * k)(*gen_ids)
        opts = (pv3d_eval_opts * k)()
        results = (pv3d_result * k)()
        keep = []
        for q, gid in enumerate(gen_ids):
            opts[q] = self._opts(int(ns[q]), int(rs[q]), 0, 0, chunk_steps, None, 0.0, 0.0, 0.0)
            res, arrays = self._alloc(gid, 0, 0, outputs, device)
            results[q] = res
            keep.append(arrays)
        self._check(self.lib.pv3d_evaluate_batch(self.h, k, ids, opts, results))
        for q in range(k):
            keep[q].update(tests=results[q].tests, latency_ms=results[q].latency_ms, waves=results[q].waves)
        return keep

    def release(self, scene_or_gen_id: int):
        self._check(self.lib.pv3d_release(self.h, scene_or_gen_id))
        self._gens.pop(scene_or_gen_id, None)


def pv3d_module_shade_noalloc(tri_xyz, module: dict, sun_xyz, samples_per_side: int, map_res: int, cell_counts,
                              stream=None) -> int:
    """pv3d_module_shade_noalloc (no device allocation inside the library).

    ``tri_xyz``: CUDA tensor, 9 float32 per triangle; ``cell_counts``: CUDA
    tensor of cells_u * cells_v int32/uint32 (overwritten); ``module``: dict with
    origin, u, v, pitch, cells_u, cells_v; ``sun_xyz``: 3 floats.  Returns the
    status code (0 = queued on ``stream``)."""
    import torch
    lib = load()
    n_cells = int(module["cells_u"]) * int(module["cells_v"])
    if tri_xyz is not None and tri_xyz.numel():
        if not (isinstance(tri_xyz, torch.Tensor) and tri_xyz.is_cuda and tri_xyz.dtype == torch.float32
                and tri_xyz.is_contiguous() and tri_xyz.numel() % 9 == 0):
            raise ValueError("tri_xyz must be a contiguous float32 CUDA tensor of 9 floats per triangle")
    if not (isinstance(cell_counts, torch.Tensor) and cell_counts.is_cuda
            and cell_counts.dtype in (torch.int32, getattr(torch, "uint32", torch.int32))
            and cell_counts.is_contiguous() and cell_counts.numel() >= n_cells):
        raise ValueError(f"cell_counts must be a contiguous int32/uint32 CUDA tensor of at least {n_cells} elements")
    if tri_xyz is not None and tri_xyz.numel() and tri_xyz.device != cell_counts.device:
        raise ValueError("tri_xyz and cell_counts must be on the same device")
    md = pv3d_module()
    md.origin[:] = [float(x) for x in module["origin"]]
    md.u[:] = [float(x) for x in module["u"]]
    md.v[:] = [float(x) for x in module["v"]]
    md.pitch = float(module["pitch"])
    md.cells_u = int(module["cells_u"]); md.cells_v = int(module["cells_v"])
    md.layout = 0; md.tracker = -1; md.string_id = 0
    sun = np.ascontiguousarray(sun_xyz, np.float64).reshape(3)
    n_tris = int(tri_xyz.numel() // 9) if tri_xyz is not None else 0
    tp = tri_xyz.data_ptr() if n_tris else None
    return lib.pv3d_module_shade_noalloc(tp, n_tris, C.byref(md), _p(sun), int(samples_per_side), int(map_res),
                                         cell_counts.data_ptr(), stream)


def raster_peak(device: int = 0) -> dict:
    """pv3d_raster_peak: measured shared-memory atomicMin throughput (the
    rasteriser's roofline) of ``device``, in G updates/s."""
    lib = load()
    a, ms = C.c_double(), C.c_double()
    rc = lib.pv3d_raster_peak(int(device), C.byref(a), C.byref(ms))
    if rc != PV3D_OK:
        raise PV3DError(rc, "pv3d_raster_peak failed")
    return {"g_atomics_per_s": a.value / 1e9, "best_ms": ms.value}


def load_workload(ctx: Context, w) -> int:
    """Load a scenes.Workload (scene, generator, sun, poses) into ``ctx``; returns the generator id."""
    sid = ctx.scene_load(w.scene.verts, w.scene.tris)
    gid = ctx.generator_define(sid, w.gen)
    ctx.set_sun(gid, w.sun.xyz, w.sun.dni, w.sun.dhi, w.sun.dt_h)
    if w.poses is not None and w.gen.pivots.shape[0] > 0:
        ctx.set_poses(gid, w.poses)
    return gid
