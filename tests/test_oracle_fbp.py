"""Property pins of the oracle's FBP surface ROS and the ellipse of Eqs. (1)-(4).

The FBP equations themselves are not printed in the paper and their
publication is not available here, so their constants stay "parity
unpinned"; what is pinned are the properties the paper and the mathematics
fix: circle without wind or slope, symmetry about the head direction
(assumption A2), the relations between HROS, BROS, FROS, LB, a and e of
Sec. 3.7, the slope-equivalent-wind round trip, the M1 limits and the
build-up effect at BUI0.
"""
import math

import numpy as np
import pytest

import oracle
from c2f_synth import FUEL_CODES

FUELS = ["C1", "C2", "C3", "C4", "C5", "C6", "C7", "D1", "M1", "M2", "O1a", "O1b",
         "S1", "S2", "S3"]
ULP = 2.0 ** -52


@pytest.mark.parametrize("fuel", FUELS)
def test_no_wind_no_slope_is_a_circle(fuel):
    r = oracle.fbp_cell(FUEL_CODES[fuel], 0.0, 123.0, 0.0, 270.0, 90.0, 80.0)
    assert r["lb"] == 1.0 and r["e"] == 0.0
    assert r["hros"] == r["bros"] and r["wse"] == 0.0
    assert np.all(r["ros8"] == r["a"]) and r["a"] == r["hros"]


@pytest.mark.parametrize("fuel", FUELS)
@pytest.mark.parametrize("wd", [270.0, 90.0, 0.0, 180.0])
def test_mirror_symmetry_about_axis_aligned_head(fuel, wd):
    """Wind along a grid axis, flat ground: ROS on axes mirrored about the head are equal."""
    r = oracle.fbp_cell(FUEL_CODES[fuel], 0.0, 0.0, 25.0, wd, 91.0, 70.0)
    head = {270.0: 0, 180.0: 2, 90.0: 4, 0.0: 6}[wd]
    ros = r["ros8"]
    for d in (1, 2, 3):
        assert ros[(head + d) % 8] == ros[(head - d) % 8]
    # Eq. (1): head axis a(1+e), back half a(1-e^2)
    a, e = r["a"], r["e"]
    assert abs(ros[head] - a * (1 + e)) <= 4 * ULP * ros[head]
    for d in (2, 3, 4):
        assert ros[(head + d) % 8] == a * (1 - e * e)


def test_rotating_the_wind_rotates_the_ros_exactly():
    base = oracle.fbp_cell(1, 0.0, 0.0, 18.0, 270.0, 90.0, 80.0)["ros8"]     # head east
    north = oracle.fbp_cell(1, 0.0, 0.0, 18.0, 180.0, 90.0, 80.0)["ros8"]    # head north
    assert np.array_equal(np.roll(base, 2), north)


@pytest.mark.parametrize("fuel", ["C1", "C2", "D1", "M1", "O1a", "S1"])
def test_ellipse_relations_sec_3_7(fuel):
    r = oracle.fbp_cell(FUEL_CODES[fuel], 12.0, 40.0, 22.0, 250.0, 92.0, 90.0)
    H, B, LB = r["hros"], r["bros"], r["lb"]
    assert abs(r["fros"] - (H + B) / (2 * LB)) <= 2 * ULP * r["fros"]      # FROS = (H+B)/(2 LB)
    assert abs(r["a"] - (H + B) / 2) <= ULP * r["a"]                       # Eq. (2)
    e4 = math.sqrt(1 - (r["fros"] / ((H + B) / 2)) ** 2)                   # Eq. (4) with t = 1
    assert abs(r["e"] - e4) <= 1e-13
    assert H >= B > 0 and LB >= 1.0
    assert abs(math.hypot(r["ux"], r["uy"]) - 1.0) <= 4 * ULP


def test_slope_equivalent_wind_round_trip():
    """No wind, slope only: the slope-equivalent wind reproduces RSF = RSZ * SF."""
    for fuel in ("C2", "C3", "C6", "D1", "S1"):
        gs = 25.0
        flat = oracle.fbp_cell(FUEL_CODES[fuel], 0.0, 0.0, 0.0, 0.0, 90.0, 80.0)["hros"]
        slp = oracle.fbp_cell(FUEL_CODES[fuel], gs, 0.0, 0.0, 0.0, 90.0, 80.0)
        sf = math.exp(3.533 * (gs / 100.0) ** 1.2)
        assert abs(slp["hros"] / flat - sf) <= 1e-12 * sf, fuel
        assert slp["wse"] > 0


def test_upslope_is_the_head_direction():
    # aspect is the downslope azimuth; aspect 270 (facing west) -> upslope east
    r = oracle.fbp_cell(FUEL_CODES["C2"], 30.0, 270.0, 0.0, 0.0, 90.0, 80.0)
    assert r["ux"] == pytest.approx(1.0, abs=1e-15) and abs(r["uy"]) < 1e-15
    assert r["ros8"][0] == max(r["ros8"])


def test_m1_limits():
    # PC = 100 gives C2, PC = 0 gives D1 (BUI at each fuel's BUI0 so BE = 1)
    for ws, gs in ((0.0, 0.0), (20.0, 0.0), (15.0, 20.0)):
        m1 = oracle.fbp_cell(FUEL_CODES["M1"], gs, 30.0, ws, 240.0, 90.0, 50.0, m1_pc=100.0)
        c2 = oracle.fbp_cell(FUEL_CODES["C2"], gs, 30.0, ws, 240.0, 90.0, 64.0)
        assert m1["hros"] == c2["hros"] and np.array_equal(m1["ros8"], c2["ros8"])
        m0 = oracle.fbp_cell(FUEL_CODES["M1"], gs, 30.0, ws, 240.0, 90.0, 50.0, m1_pc=0.0)
        d1 = oracle.fbp_cell(FUEL_CODES["D1"], gs, 30.0, ws, 240.0, 90.0, 32.0)
        assert m0["hros"] == d1["hros"] and np.array_equal(m0["ros8"], d1["ros8"])


def test_buildup_effect():
    # O1 has no build-up effect; other fuels are monotone in BUI and BE(BUI0) = 1
    o_lo = oracle.fbp_cell(FUEL_CODES["O1a"], 0.0, 0.0, 10.0, 270.0, 90.0, 20.0)
    o_hi = oracle.fbp_cell(FUEL_CODES["O1a"], 0.0, 0.0, 10.0, 270.0, 90.0, 150.0)
    assert o_lo["hros"] == o_hi["hros"]
    c1 = [oracle.fbp_cell(1, 0.0, 0.0, 10.0, 270.0, 90.0, b)["hros"] for b in (40, 72, 120)]
    assert c1[0] < c1[1] < c1[2]
    # log-linear in 1/BUI: BE(b1) BE(b2) = BE(b3) when 1/b1 + 1/b2 = 1/b3 + 1/72
    b1, b2 = 40.0, 120.0
    b3 = 1.0 / (1 / b1 + 1 / b2 - 1 / 72.0)
    h = lambda b: oracle.fbp_cell(1, 0.0, 0.0, 10.0, 270.0, 90.0, b)["hros"]
    assert abs(h(b1) * h(b2) / (h(72.0) * h(b3)) - 1.0) < 1e-13


def test_rsi_saturates_at_a():
    # RSI = a (1 - exp(-b ISI))^c rises toward a (BE = 1 at BUI0) and never exceeds it
    prev = 0.0
    for ffmc in (85.0, 92.0, 97.0, 100.9):
        h = oracle.fbp_cell(FUEL_CODES["C2"], 0.0, 0.0, 400.0, 270.0, ffmc, 64.0)["hros"]
        assert prev < h < 110.0
        prev = h
    assert 110.0 - prev < 0.3


def test_wind_speeds_up_the_head_and_stretches_the_ellipse():
    prev = None
    for ws in (0, 5, 10, 20, 40, 60):
        r = oracle.fbp_cell(1, 0.0, 0.0, float(ws), 270.0, 90.0, 80.0)
        if prev is not None:
            assert r["hros"] > prev["hros"] and r["lb"] > prev["lb"]
        prev = r


def test_centre_offset_ellipse_mode_hits_head_and_back():
    r = oracle.fbp_cell(1, 0.0, 0.0, 20.0, 270.0, 90.0, 80.0, ellipse_mode=1)
    assert abs(r["ros8"][0] - r["hros"]) <= 1e-15 * r["hros"] * 8
    assert abs(r["ros8"][4] - r["bros"]) <= 1e-12 * r["hros"]
    assert r["ros8"][1] == r["ros8"][7] and r["ros8"][2] == r["ros8"][6]
