"""Helpers that run the CUDA path and the FP64 oracle on the same seeded
workload and compare them with the acceptance criteria:

* shaded flags agree on >= 99.9 % of the samples the oracle does not mask
  (ray within one texel of a triangle edge, or a depth gap below the texel-scale
  swing; back-lit and grazing modules are masked whole);
* cell shaded fractions differ by at most 1/n^2 beyond the cell's masked samples;
* annual (or evaluated-period) energy loss differs by at most 0.1 % absolute.
"""
from __future__ import annotations

import numpy as np

import oracle

FLAG_AGREEMENT = 0.999
LOSS_PP = 0.1


def run_gpu(ctx, gid, w, step_begin=0, step_end=0, outputs=("energy", "energy_unshaded", "power",
                                                                   "power_unshaded", "sample_bits", "cell_counts"),
            chunk_steps=0, device=True, path=0, window_groups=0, map_res=0):
    import torch
    r = ctx.evaluate(gid, n=w.n, map_res=map_res or w.map_res, step_begin=step_begin, step_end=step_end,
                     chunk_steps=chunk_steps, outputs=outputs, device=device, path=path,
                     window_groups=window_groups)
    if device:
        torch.cuda.synchronize()
    out = {}
    for k, v in r.items():
        if hasattr(v, "cpu"):
            a = v.cpu().numpy()
            if k == "sample_bits":
                a = a.view(np.uint64)
            out[k] = a
        else:
            out[k] = v
    return out


def module_cell_slices(gen):
    cells = gen.cells_u.astype(np.int64) * gen.cells_v
    starts = np.concatenate([[0], np.cumsum(cells)])
    return starts


def compare(w, g, o, steps_rel, modules=None):
    """Compare GPU results ``g`` (rows = steps of its evaluated range) with the
    oracle result ``o`` evaluated on ``steps_rel`` (row indices into g) and the
    oracle's module list.  Returns a dict of statistics."""
    n = w.n
    starts = module_cell_slices(w.gen)
    mods = o["modules"]
    cols = np.concatenate([np.arange(starts[m], starts[m + 1]) for m in mods])
    gb = oracle.unpack_bits(g["sample_bits"][steps_rel][:, cols], n)
    ob = oracle.unpack_bits(o["bits"], n)
    mk = oracle.unpack_bits(o["mbits"], n)
    lit = (w.sun.xyz[o["steps"], 2] > 0)
    gb, ob, mk = gb[lit], ob[lit], mk[lit]
    unm = ~mk
    n_unm = int(unm.sum())
    agree = (gb == ob)[unm].mean() if n_unm else 1.0
    # cell fractions beyond masked samples
    gcnt = gb.sum(-1).astype(np.int64)
    ocnt = ob.sum(-1).astype(np.int64)
    slack = mk.sum(-1) + 1
    cell_ok = (np.abs(gcnt - ocnt) <= slack).mean() if gcnt.size else 1.0
    return dict(agree=float(agree), n_unmasked=n_unm, n_total=int(mk.size), masked_frac=float(mk.mean()) if mk.size else 0.0,
                cell_ok=float(cell_ok), n_disagree=int(((gb != ob) & unm).sum()))


def energy_checks(w, g, o, steps_rel, loss_slack=LOSS_PP):
    """Energy-side parity, sample by sample:
    1. the GPU's per-step module power equals the oracle's PV model applied to
       the GPU's own cell counts (the reduction and electrical model are exact
       up to FP32 rounding);
    2. the GPU's power lies between the oracle's power with every masked
       sample forced lit and forced shaded (P is non-increasing in each flag),
       for every (step, module) whose unmasked flags agree; and the loss over
       the evaluated steps lies in the same envelope, within ``loss_slack``.
    """
    n = w.n
    starts = module_cell_slices(w.gen)
    mods = o["modules"]
    cols = np.concatenate([np.arange(starts[m], starts[m + 1]) for m in mods])
    steps = o["steps"]
    gcnt = g["cell_counts"][steps_rel][:, cols].astype(np.int32)
    pg = g["power"][steps_rel][:, mods].astype(np.float64)
    pc = oracle.power_from_counts(w, steps, mods, gcnt)
    assert np.all(np.abs(pg - pc) <= 1e-4 * np.maximum(np.abs(pc), 1.0) + 1e-3), np.abs(pg - pc).max()
    ob, mb = o["bits"], o["mbits"]
    lo = oracle.power_from_counts(w, steps, mods, oracle.popcount64(ob | mb))   # masked -> shaded
    hi = oracle.power_from_counts(w, steps, mods, oracle.popcount64(ob & ~mb))  # masked -> lit
    gb = g["sample_bits"][steps_rel][:, cols]
    cell_bad = ((gb ^ ob) & ~mb) != 0
    # (step, module) pairs whose unmasked flags all agree
    mod_of_col = np.repeat(np.arange(len(mods)), np.diff(starts)[mods])
    bad = np.zeros(pg.shape, bool)
    np.logical_or.at(bad, (slice(None), mod_of_col), cell_bad)
    tol = 1e-4 * np.maximum(np.abs(hi), 1.0) + 1e-3
    ok = (pg >= lo - tol) & (pg <= hi + tol)
    assert ok[~bad].all(), (np.argwhere(~ok & ~bad)[:5], pg[~ok & ~bad][:5], lo[~ok & ~bad][:5], hi[~ok & ~bad][:5])
    dt = w.sun.dt_h[steps].astype(np.float64)[:, None]
    pu = o["power_unshaded"]
    eu = float((pu * dt).sum())
    if eu > 0:
        l_g = 100 * (1 - float((pg * dt).sum()) / eu)
        l_min = 100 * (1 - float((hi * dt).sum()) / eu)
        l_max = 100 * (1 - float((lo * dt).sum()) / eu)
        assert l_min - loss_slack <= l_g <= l_max + loss_slack, (l_min, l_g, l_max)
        return dict(loss_gpu=l_g, loss_min=l_min, loss_max=l_max, bad_pairs=int(bad.sum()))
    return dict(bad_pairs=int(bad.sum()))


def loss_pp(e, eu):
    e = float(np.sum(e)); eu = float(np.sum(eu))
    return 0.0 if eu <= 0 else 100.0 * (1.0 - e / eu)
