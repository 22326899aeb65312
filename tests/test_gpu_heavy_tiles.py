"""GPU parity on the tile kernels' less common paths: tiles handed from one
warp per tile to one block per tile (a block-wide sample-driven test, or a
shared-memory depth tile and the test of its samples, whichever is estimated
cheaper) because they keep more than 64 triangles, have more than 512 binned
triangles, or more than 16 or 64 receiver modules (receivers then staged in
chunks, without plane culling); 32-texel tiles go on with more than 64
binned triangles.
Each case must agree with the FP64 oracle, be bit-identical to the map path
(HBM shadow map + gather), and the work counters must show that the intended
path ran."""
import numpy as np
import pytest

import oracle
from paper_1410_5780_gb300 import pv3d, scenes as S

from parity import FLAG_AGREEMENT, compare, energy_checks, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case,tile,map_res,tiny,cells", [
    ("block_kept", 64, 256, False, 30),        # kept > 64: one block, shared-memory raster
    ("block_raster", 64, 128, False, 60),      # binned > 512: one block, shared-memory raster
    ("many_receivers", 64, 128, True, 30),     # > 16 receivers per tile: one block
    ("receiver_chunks", 64, 64, True, 30),     # > 64 receivers: staged in chunks, no plane culling, raster
    ("warp_tiles", 32, 512, False, 30),        # the same canopy on small tiles
    ("block_raster_128", 128, 256, False, 60), # 128-texel tiles: block raster of a 64 KB shared tile
    ("crowded_32", 32, 128, False, 60),        # 32-texel tiles, > 64 binned: handed on before the keep loop
])
def test_heavy_tile_paths(case, tile, map_res, tiny, cells):
    w = S.make_canopy(31 if not tiny else 32, tiny_modules=tiny, map_res=map_res, cells=cells)
    o = oracle.evaluate_workload(w)
    with pv3d.Context(device=0, tile=tile) as c:
        gid = pv3d.load_workload(c, w)
        g = run_gpu(c, gid, w)
        st = compare(w, g, o, np.arange(w.sun.n_steps))
        assert st["agree"] >= FLAG_AGREEMENT, (case, st)
        assert st["cell_ok"] == 1.0, (case, st)
        energy_checks(w, g, o, np.arange(w.sun.n_steps))
        m = run_gpu(c, gid, w, path=pv3d.PV3D_PATH_MAP)
        for k in ("sample_bits", "cell_counts", "power", "energy"):
            np.testing.assert_array_equal(g[k], m[k], err_msg=f"{case}: {k}")
        assert g["cell_counts"].sum() > 0
        c.evaluate(gid, n=w.n, map_res=w.map_res, profile=3)
        p = c.last_profile()
    why = p["heavy_why"]  # [receivers, binned triangles, kept triangles]
    p = {k: v for k, v in p.items() if not k.endswith("_ms")}
    warp_tiles = p["nonempty_tiles"] - p["heavy_tiles"]
    raster_tiles = p["nonempty_tiles"] - p["sample_tiles"]
    if case == "block_kept":
        assert why[2] > 0 and p["heavy_tiles"] > 0, p
    elif case == "crowded_32":
        # handed on for their binned count (more than a warp keeps), rasterised
        assert why[1] > 0 and p["heavy_tiles"] > 0 and p["texel_visits"] > 0, p
    elif case in ("block_raster", "block_raster_128"):
        assert why[1] > 0 and raster_tiles > 0 and p["texel_visits"] > 0, p
    elif case == "many_receivers":
        assert why[0] > 0 and raster_tiles > 0, p
    elif case == "receiver_chunks":
        # one tile holds every module; without plane culling it keeps the
        # whole canopy and is rasterised, its receivers staged in chunks
        assert why[0] > 0 and raster_tiles > 0, p
    else:
        assert warp_tiles > 0, p
