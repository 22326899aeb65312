"""Checks against the few numbers the paper prints (tests/golden/paper_figures.json)."""
import json
import math
import os

import numpy as np

import oracle
from paper_1410_5780_gb300 import scenes as S

with open(os.path.join(os.path.dirname(__file__), "golden", "paper_figures.json")) as f:
    PAPER = json.load(f)


def test_daylight_steps_per_year_at_ten_minutes():
    """Section 4: a year of daylight moments at 10-min resolution is ~26,000 steps."""
    for lat in (0.0, 40.0, 52.4):
        sun = S.year_sun(lat, PAPER["time_step_minutes_recommended"] / 60.0)
        ref = PAPER["section4"]["daylight_steps_10min_year"]
        assert abs(sun.n_steps - ref) / ref < 0.03


def test_section4_evaluation_count():
    """Section 4: 80,000 triangles x 26,000 steps x 1,400 areas ~ 3e12."""
    s3 = PAPER["section3_1"]
    areas = s3["panels"] * s3["cells_per_panel"] * PAPER["section4"]["areas_per_cell"]
    assert abs(areas - PAPER["section4"]["areas_whole_generator"]) / 1400 < 0.01
    ev = s3["triangles"] * PAPER["section4"]["daylight_steps_10min_year"] * areas
    assert abs(ev - PAPER["section4"]["shading_evaluations"]) / 3e12 < 0.05


def test_fig2_module_one_shaded_cell():
    """Fig. 2 module (36 cells, 2 bypass diodes): one beam-shaded cell either
    bypasses its 18-cell substring or limits the whole module's current."""
    f2 = PAPER["fig2_generator"]
    cells, diodes = f2["cells_per_module"], f2["bypass_diodes"]
    lay = S.standard_layout(4, cells // 4, diodes)
    assert np.bincount(lay.cell_sub).tolist() == [cells // diodes] * diodes
    vk = cells // diodes * oracle.V_CELL
    for g_full, g_diff in [(1000.0, 100.0), (700.0, 450.0)]:
        g = np.full(cells, g_full)
        g[5] = g_diff
        i_full, i_diff = (oracle.I_REF * x / 1000.0 for x in (g_full, g_diff))
        expect = max(i_full * (vk - oracle.V_DIODE), i_diff * 2 * vk)
        assert math.isclose(oracle.module_pmpp(g, lay.cell_sub, diodes), expect, rel_tol=1e-12)


def test_three_by_three_areas_are_cell_centred():
    """Section 2 step 3: 3x3 areas per cell; for n = 1 the sample is the cell centre."""
    assert PAPER["areas_per_cell_recommended"] == 9
    w = S.make_tiny()
    c1 = oracle.samples(w.gen, None, 0, 0, 1)
    c3 = oracle.samples(w.gen, None, 0, 0, 3).reshape(-1, 9, 3)
    assert np.allclose(c3.mean(1), c1, atol=1e-9)
    assert np.allclose(c3[:, 4], c1, atol=1e-9)  # the middle area is centred on the cell
