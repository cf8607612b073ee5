"""The oracle's rate-of-spread rows against a plain high-precision evaluation.

The oracle (like the GPU library) evaluates the FBP chain and the ellipse of
Sec. 3.7 / Eq. (1) with its own table-driven exp and log, rounded reciprocals
of per-fuel and per-hour divisors and half-integer power shortcuts.  Here the
same formulas are evaluated the plain way (true divisions, x ** y, mpmath at
120 bits; ``tests/fbp_plain.py``) and every output of the oracle's row --
HROS, BROS, LB, FROS, a, e, the head direction, WSV, WSE and the 8 axis rates
-- must agree within 1e-12 relative (the table tolerance), for every fuel
code, on both sides of each switch of the chain: the 40 km/h wind-function
switch, WSE above 40 (its formula and its 112.45 cap), the ISF guard, the
curing switch at 58.8 %, the O1 LB switch at WSV = 1, flat and sloped cells
(slopes at and beyond the 60 % cap), M1 / M2 at 0, 35 and 100 % conifer, and
both ellipse modes.

What this pins: the arithmetic and the branch structure of the oracle's row.
What it cannot pin: the FBP coefficient values and equation edition, which
neither the paper nor this repository holds a publication copy of (the plain
evaluation uses the same constants).
"""
import itertools
import math

import pytest

import fbp_plain as P
import oracle

mpmath = pytest.importorskip("mpmath")

# hourly weather (ws km/h, wind from deg, FFMC, BUI): the workloads' ranges,
# calm, the 40 km/h switch (WSV exactly 40 on flat ground), just above it,
# strong wind, very dry fuel, and WSV exactly 1 and below 1 (O1 LB switch)
WEATHERS = [(0.0, 270.0, 90.0, 80.0), (20.0, 270.0, 90.0, 80.0), (15.0, 30.0, 85.0, 40.0),
            (35.0, 200.0, 93.0, 120.0), (40.0, 270.0, 90.0, 80.0), (40.5, 270.0, 90.0, 80.0),
            (55.0, 135.0, 88.0, 60.0), (10.0, 0.0, 96.0, 150.0), (1.0, 270.0, 90.0, 80.0),
            (0.5, 270.0, 90.0, 80.0)]
# (slope %, aspect deg): flat, gentle, steep, at the 60 % cap, beyond it
TOPO = [(0.0, 0.0), (10.0, 45.0), (35.0, 300.0), (60.0, 180.0), (80.0, 90.0)]
# (M1/M2 percent conifer, O1 curing %): default, and both sides of the switches
MIX = [(50.0, 60.0), (0.0, 30.0), (35.0, 58.8), (100.0, 100.0), (50.0, 58.7)]

REL = 1e-12
POSITIVE = ("hros", "bros", "lb", "fros", "a")     # relative error
UNIT = ("e", "ux", "uy")                            # bounded by 1: absolute error
SPEEDS = ("wsv", "wse")                             # relative, absolute near 0 (km/h)


def _close(got, want, field):
    got, want = float(got), float(want)
    if field in UNIT:
        return abs(got - want) <= REL
    floor = 1.0 if field in SPEEDS else 1e-300
    return abs(got - want) <= REL * max(abs(want), floor)


def _cases():
    for fuel in range(1, 16):
        mixes = MIX if fuel in (P.M1, P.M2, P.O1A, P.O1B) else MIX[:1]
        for (pc, cur), w, t, mode in itertools.product(mixes, WEATHERS, TOPO, (0, 1)):
            yield fuel, t, w, pc, cur, mode


@pytest.fixture(scope="module")
def mp():
    return P.mp_backend()


def test_oracle_row_equals_plain_evaluation_within_1e12(mp):
    bad, branches, n = [], {}, 0
    for fuel, (gs, asp), (ws, wd, ff, bui), pc, cur, mode in _cases():
        o = oracle.fbp_cell(fuel, gs, asp, ws, wd, ff, bui, m1_pc=pc, o1_curing=cur, ellipse_mode=mode)
        p = P.fbp_row(mp, fuel, gs, asp, ws, wd, ff, bui, pc, cur, mode)
        n += 1
        for k, v in p["branch"].items():
            branches.setdefault(k, set()).add(v)
        for f in POSITIVE + UNIT + SPEEDS:
            if not _close(o[f], p[f], f):
                bad.append((fuel, gs, asp, ws, wd, ff, bui, pc, cur, mode, f, o[f], float(p[f])))
        for k in range(8):
            if not _close(o["ros8"][k], p["ros8"][k], "ros"):
                bad.append((fuel, gs, asp, ws, wd, ff, bui, pc, cur, mode, k, o["ros8"][k],
                            float(p["ros8"][k])))
    assert not bad, (len(bad), bad[:5])
    assert n > 2000
    # both sides of every switch of the chain were exercised
    assert branches["wind_high"] == {False, True}
    assert branches["sloped"] == {False, True}
    assert branches["curing_low"] == {False, True}
    assert branches["o1_wsv_ge_1"] == {False, True}
    assert branches["wse_high"] == {"formula", "cap"}
    assert branches["isf_guard"] == {True}


def test_libm_plain_evaluation_is_within_5e13_of_mpmath(mp):
    """The GPU twin of this test compares the GPU's table rows with the plain
    evaluation in binary64 (libm); that evaluation is itself within 5e-13 of
    the 120-bit one (its worst case, 3e-13, is a mode-1 rate across a strong
    wind), with the back half of the mode-1 ray multiplied out by its
    conjugate (the written form cancels there)."""
    worst = 0.0
    for fuel, (gs, asp), (ws, wd, ff, bui), pc, cur, mode in _cases():
        p = P.fbp_row(mp, fuel, gs, asp, ws, wd, ff, bui, pc, cur, mode)
        q = P.fbp_row(P.LIBM, fuel, gs, asp, ws, wd, ff, bui, pc, cur, mode, conjugate_back=True)
        for f in ("hros", "bros", "lb", "fros", "a"):
            worst = max(worst, abs(q[f] - float(p[f])) / max(abs(float(p[f])), 1e-300))
        for k in range(8):
            worst = max(worst, abs(q["ros8"][k] - float(p["ros8"][k])) / max(abs(float(p["ros8"][k])), 1e-300))
    assert worst < 5e-13, worst


def test_conjugate_back_half_is_the_same_ray(mp):
    """r = b^2 (a^2 - c^2) / (a b sqrt(Q) - b^2 c cos) is the written ray
    multiplied out by the conjugate of its numerator (a^2 - c^2 = HROS BROS):
    at 120 bits the two forms agree to 1e-25 on every back-half axis."""
    for fuel, (gs, asp), (ws, wd, ff, bui), pc, cur, _ in itertools.islice(_cases(), 0, None, 7):
        p = P.fbp_row(mp, fuel, gs, asp, ws, wd, ff, bui, pc, cur, 1)
        q = P.fbp_row(mp, fuel, gs, asp, ws, wd, ff, bui, pc, cur, 1, conjugate_back=True)
        for k in range(8):
            assert abs(p["ros8"][k] - q["ros8"][k]) <= mpmath.mpf(1e-25) * abs(p["ros8"][k]) + mpmath.mpf(1e-60)


def test_plain_evaluation_meets_the_closed_forms(mp):
    """The plain evaluation itself against facts that do not depend on it:
    the ellipse relations of Sec. 3.7 (a = (H + B)/2, FROS = (H + B)/(2 LB),
    e = sqrt(1 - 1/LB^2)), Eq. (1) at the head a (1 + e), the ray of mode 1
    hitting H ahead and B behind, and the circle at no wind and no slope."""
    p = P.fbp_row(mp, 2, 0.0, 0.0, 25.0, 270.0, 90.0, 80.0)
    assert abs(p["a"] - (p["hros"] + p["bros"]) / 2) < 1e-30
    assert abs(p["fros"] - (p["hros"] + p["bros"]) / (2 * p["lb"])) < 1e-30
    assert abs(p["e"] ** 2 - (1 - 1 / p["lb"] ** 2)) < 1e-30
    assert abs(p["ros8"][0] - p["a"] * (1 + p["e"])) < 1e-28     # head east, Eq. (1)
    r = P.fbp_row(mp, 2, 0.0, 0.0, 25.0, 270.0, 90.0, 80.0, ellipse_mode=1)
    assert abs(r["ros8"][0] - r["hros"]) < 1e-28 and abs(r["ros8"][4] - r["bros"]) < 1e-28
    c = P.fbp_row(mp, 1, 0.0, 0.0, 0.0, 270.0, 90.0, 80.0)
    assert abs(c["hros"] - c["bros"]) < 1e-30 and c["lb"] == 1
    assert all(abs(x - c["hros"]) < 1e-30 for x in c["ros8"])
