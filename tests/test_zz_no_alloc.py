"""pv3d_module_shade_noalloc against pv3d_evaluate.

The no-allocation entry point serves callers that cannot allocate device
memory while they run (their own memory pool owns the GPU, a latency-critical
loop cannot take cudaMalloc's synchronisation, or the work is being recorded
into a stream capture).  Its results must match the regular evaluation of the
same one-module generator within the parity tolerance: per cell at most one
sample (1/n^2 of the cell's fraction) apart, and at most 0.1 % of all samples
different.  Two calls in a row share the library's fixed shadow map, so the
second call also checks that each call clears what it uses.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from paper_1410_5780_gb300 import pv3d, scenes as S

pytestmark = pytest.mark.gpu


def _one_module_workload():
    w = S.make_tiny(day=355, n=4, map_res=1024)
    keep = [1]
    g = w.gen
    w.gen = S.Generator(origin=g.origin[keep], u=g.u[keep], v=g.v[keep], cells_u=g.cells_u[keep],
                        cells_v=g.cells_v[keep], pitch=g.pitch[keep], layout=g.layout[keep],
                        tracker=g.tracker[keep], string=g.string[keep], layouts=g.layouts, pivots=g.pivots)
    # a few more occluders so that several steps are partly shaded
    mb = S.MeshBuilder()
    mb.add(w.scene.verts, w.scene.tris)
    mb.beam((1.5, -1.5, 0.0), (1.5, -1.5, 2.5), 0.2)
    mb.box((-2.5, -2.0, 0.0), (-1.8, -1.6, 1.8))
    w.scene = mb.build()
    return w


def test_noalloc_matches_evaluate_on_consecutive_calls():
    import torch
    pv3d.load(build_if_missing=True)
    w = _one_module_workload()
    lit = np.flatnonzero(w.sun.xyz[:, 2] > 0)
    with pv3d.Context(device=0, map_res=w.map_res) as ctx:
        gid = pv3d.load_workload(ctx, w)
        r = ctx.evaluate(gid, n=w.n, map_res=w.map_res, outputs=("cell_counts",), device=True)
        torch.cuda.synchronize()
        ref = r["cell_counts"].cpu().numpy().astype(np.int64)
    assert ref.sum() > 0
    tri = torch.tensor(w.scene.verts[w.scene.tris].reshape(-1, 9), dtype=torch.float32, device="cuda:0")
    m = w.gen
    module = dict(origin=m.origin[0], u=m.u[0], v=m.v[0], pitch=float(m.pitch[0]), cells_u=int(m.cells_u[0]),
                  cells_v=int(m.cells_v[0]))
    counts = torch.empty(int(m.cells_u[0] * m.cells_v[0]), dtype=torch.int32, device="cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    nn = w.n * w.n
    checked = 0
    for st in list(lit) + [int(lit[len(lit) // 2])]:  # consecutive calls, the last repeats a step
        rc = pv3d.pv3d_module_shade_noalloc(tri, module, w.sun.xyz[st], w.n, w.map_res, counts, stream)
        assert rc == pv3d.PV3D_OK
        torch.cuda.synchronize()
        got = counts.cpu().numpy().astype(np.int64)
        diff = np.abs(got - ref[st])
        assert diff.max() <= 1, (st, diff.max())
        assert diff.sum() <= 0.001 * got.size * nn, (st, diff.sum())
        checked += int(ref[st].sum() > 0)
    assert checked >= 3


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    pv3d.load(build_if_missing=True)
    w = _one_module_workload()
    m = w.gen
    module = dict(origin=m.origin[0], u=m.u[0], v=m.v[0], pitch=float(m.pitch[0]), cells_u=int(m.cells_u[0]),
                  cells_v=int(m.cells_v[0]))
    tri = torch.tensor(w.scene.verts[w.scene.tris].reshape(-1, 9), dtype=torch.float32, device="cuda:0")
    counts = torch.empty(int(m.cells_u[0] * m.cells_v[0]), dtype=torch.int32, device="cuda:0")
    sun = w.sun.xyz[12]
    assert pv3d.pv3d_module_shade_noalloc(tri, module, sun, 4, 2 * pv3d.PV3D_NOALLOC_MAX_RES, counts) \
        == pv3d.PV3D_E_TOOBIG
    assert pv3d.pv3d_module_shade_noalloc(tri, module, sun, 4, 1000, counts) == pv3d.PV3D_E_INVALID
    assert pv3d.pv3d_module_shade_noalloc(tri, module, sun * 1.01, 4, 1024, counts) == pv3d.PV3D_E_INVALID
