"""GPU rate-of-spread table rows against the plain evaluation (needs a GB300).

Twin of tests/test_oracle_fbp_plain.py: the table kernel's HROS and 8 axis
rates (c2f_get_ros), for every fuel code on flat, sloped and capped-slope
cells, under weather on both sides of the wind and O1 switches, M1 / M2 mixes
and curing on both sides of 58.8 %, in both ellipse modes, must agree with the
straightforward binary64 evaluation of the same formulas (true divisions,
libm exp / log / pow; ``tests/fbp_plain.py``) within 1e-12 relative.  That
evaluation is itself within 5e-13 of a 120-bit one (checked on the CPU), so
this bounds the GPU's error against the exact rates by 1.5e-12 without
needing mpmath on the GPU machine.
"""
import numpy as np
import pytest

import fbp_plain as P
import paper_1905_09317_gb300 as c2f
from test_oracle_fbp_plain import MIX, TOPO, WEATHERS

pytestmark = pytest.mark.gpu


def test_gpu_rows_equal_plain_evaluation_within_1e12():
    c2f.build()
    fuels = np.arange(1, 16, dtype=np.uint8)
    rows, cols = len(TOPO), len(fuels)
    fuel = np.tile(fuels, (rows, 1))
    slope = np.array([[t[0]] * cols for t in TOPO], dtype=np.float32)
    aspect = np.array([[t[1]] * cols for t in TOPO], dtype=np.float32)
    weather = np.array(WEATHERS, dtype=np.float64)
    n = rows * cols
    bad, checked = [], 0
    with c2f.Context(0) as ctx:
        lid = ctx.load_landscape(fuel, slope, aspect, cell_size=100.0)
        ctx.set_weather(lid, weather)
        for (pc, cur) in MIX:
            for mode in (0, 1):
                p = c2f.default_params(hours=len(WEATHERS), m1_pc=pc, o1_curing_pct=cur, ellipse_mode=mode)
                for h, (ws, wd, ff, bui) in enumerate(WEATHERS):
                    ros8, hros, _ = ctx.get_ros(lid, p, h, n)
                    for cell in range(n):
                        r, c = divmod(cell, cols)
                        gs, asp = TOPO[r]
                        ref = P.fbp_row(P.LIBM, int(fuel[r, c]), gs, asp, ws, wd, ff, bui, pc, cur, mode,
                                        conjugate_back=True)
                        checked += 1
                        if abs(hros[cell] - ref["hros"]) > 1e-12 * abs(ref["hros"]):
                            bad.append(("hros", pc, cur, mode, h, cell, hros[cell], ref["hros"]))
                        for k in range(8):
                            if abs(ros8[cell, k] - ref["ros8"][k]) > 1e-12 * abs(ref["ros8"][k]):
                                bad.append(("ros", pc, cur, mode, h, cell, k, ros8[cell, k], ref["ros8"][k]))
        ctx.release(lid)
    assert checked == len(MIX) * 2 * len(WEATHERS) * n
    assert not bad, (len(bad), bad[:5])
