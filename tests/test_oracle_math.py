"""Pins of the oracle's own elementary functions and Philox generator.

The oracle computes every exp/log/sin/cos itself (so the GPU can reproduce
it bit for bit); these tests pin those functions to high-precision values
from mpmath (an independent arbitrary-precision library) and Philox to its
published known-answer vectors.
"""
import math
import os

import mpmath
import numpy as np
import pytest

import c2f_synth as S
import oracle
from conftest import ROOT

mpmath.mp.prec = 200
ULP = 2.0 ** -52


def _rel(a, b):
    b = float(b)
    return abs(a - b) / abs(b) if b != 0 else abs(a)


def test_exp_accuracy():
    xs = np.concatenate([np.linspace(-745.0, 709.7, 4001), np.linspace(-1, 1, 2001),
                         [0.0, 1e-300, -1e-300, 0.5 * math.log(2), -0.5 * math.log(2)]])
    worst = max(_rel(oracle.exp(x), mpmath.exp(mpmath.mpf(float(x)))) for x in xs
                if float(mpmath.exp(mpmath.mpf(float(x)))) > 1e-300)
    assert worst <= 2 * ULP
    assert oracle.exp(0.0) == 1.0
    assert oracle.exp(800.0) == math.inf and oracle.exp(-800.0) == 0.0


def test_log_accuracy():
    xs = np.concatenate([np.exp(np.linspace(-700, 700, 4001)), np.linspace(0.5, 2.0, 3001),
                         [1.0, 2.0, 0.5, 1e-310, 5e-324, 1.7e308]])
    for x in xs:
        ref = mpmath.log(mpmath.mpf(float(x)))
        got = oracle.log(float(x))
        if ref == 0:
            assert got == 0.0
        else:
            # relative error near 1 is bounded by the absolute error of log(m)
            assert abs(got - float(ref)) <= 2 * ULP * max(abs(float(ref)), 1.0) * 1.0001
    assert oracle.log(1.0) == 0.0
    assert oracle.log(0.0) == -math.inf and math.isnan(oracle.log(-1.0))


def test_pow_accuracy():
    rng = np.random.default_rng(0)
    for _ in range(3000):
        x = float(rng.uniform(1e-6, 100.0)); y = float(rng.uniform(-5, 5))
        ref = mpmath.power(mpmath.mpf(x), mpmath.mpf(y))
        bound = (abs(y * math.log(x)) + 3.0) * ULP
        assert _rel(oracle.pow(x, y), ref) <= bound
    assert oracle.pow(0.0, 2.155) == 0.0 and oracle.pow(0.0, 0.0) == 1.0


def test_sincos_deg_accuracy_and_exact_quadrants():
    xs = np.concatenate([np.linspace(-1000, 1000, 8001), [45.0, 135.0, 30.0, 60.0, 1e-8]])
    for x in xs:
        s, c = oracle.sincos_deg(float(x))
        rad = mpmath.mpf(float(x)) * mpmath.pi / 180
        assert abs(s - float(mpmath.sin(rad))) <= 3 * ULP
        assert abs(c - float(mpmath.cos(rad))) <= 3 * ULP
    for k in range(-12, 13):
        s, c = oracle.sincos_deg(90.0 * k)
        exp_s = [0.0, 1.0, 0.0, -1.0][k % 4]
        exp_c = [1.0, 0.0, -1.0, 0.0][k % 4]
        assert s == exp_s and c == exp_c, (k, s, c)


def test_binary32_functions():
    f32ulp = 2.0 ** -23
    for x in np.linspace(-87.0, 88.0, 3001, dtype=np.float32):
        ref = mpmath.exp(mpmath.mpf(float(x)))
        assert _rel(float(oracle.expf(x)), ref) <= 1.5 * f32ulp
    assert oracle.expf(0.0) == np.float32(1.0)
    for u in np.concatenate([np.linspace(2.0 ** -25, 1.0, 3001, dtype=np.float32),
                             np.float32([1.0, 0.5, 2.0 ** -24])]):
        ref = mpmath.log(mpmath.mpf(float(u)))
        got = float(oracle.logf(u))
        assert abs(got - float(ref)) <= 1.5 * f32ulp * max(abs(float(ref)), 1.0)
    assert oracle.logf(1.0) == 0.0
    for u in np.linspace(0.0, 1.0, 4001, dtype=np.float32):
        ref = mpmath.cos(2 * mpmath.pi * mpmath.mpf(float(u)))
        assert abs(float(oracle.cos_turnsf(u)) - float(ref)) <= 2.0 * f32ulp
    for q in range(5):
        assert oracle.cos_turnsf(q * 0.25) == [1.0, 0.0, -1.0, 0.0, 1.0][q]


def _kat():
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "philox_kat.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].split()
            if line:
                v = [int(t, 16) for t in line]
                rows.append((v[:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert oracle.philox4x32_10(ctr, key) == out


def test_noise_factor_distribution():
    """exp(sigma z) with z from Box-Muller: log f / sigma has mean 0, variance 1."""
    sig = 0.1
    z = np.array([math.log(float(oracle.noise_factor(1234, r, c, 0, sig))) / sig
                  for r in range(40) for c in range(500)])
    assert abs(z.mean()) < 0.03 and abs(z.std() - 1.0) < 0.03
    assert oracle.noise_factor(1, 2, 3, 4, 0.0) == np.float32(1.0)
    # one draw per (replica, cell, hour): changing any coordinate changes it
    a = oracle.noise_factor(7, 1, 2, 3, sig)
    assert a != oracle.noise_factor(7, 1, 2, 4, sig) and a != oracle.noise_factor(7, 2, 2, 3, sig)


def test_noise_factor_equals_a_plain_box_muller():
    """The perturbation of (replica, cell, hour): f = exp(sigma z), z by Box-Muller
    from the Philox block at counter (replica, cell, hour, 0) under the key
    (seed low word, seed high word), u = ((x >> 8) + 1/2) 2^-24 from its first two
    words, z = sqrt(-2 ln u1) cos(2 pi u2).  The oracle's binary32 value against
    the same mapping evaluated with float64 libm functions on the known-answer-
    pinned Philox block: within 2^-17 relative (binary32 rounding of u, log, sqrt,
    cos and exp, amplified by |sigma z| < 6)."""
    rng = np.random.default_rng(5)
    for _ in range(3000):
        seed = int(rng.integers(0, 2 ** 63))
        r, c, h = (int(v) for v in rng.integers(0, 2 ** 20, 3))
        sig = float(np.float32(rng.choice([0.05, 0.1, 0.5, 1.0])))
        x = oracle.philox4x32_10([r, c, h, 0], [seed & 0xFFFFFFFF, seed >> 32])
        u1 = ((x[0] >> 8) + 0.5) * 2.0 ** -24
        u2 = ((x[1] >> 8) + 0.5) * 2.0 ** -24
        z = math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)
        f_plain = math.exp(sig * z)
        f = float(oracle.noise_factor(seed, r, c, h, sig))
        assert abs(f - f_plain) <= 2.0 ** -17 * f_plain, (seed, r, c, h, sig, f, f_plain)


def test_ignition_draw_equals_its_integer_mapping():
    """A random ignition cell (ignition_mode 1): the Philox block at counter
    (replica, 0, 0, 1) under the run key, index (x0 * n_burnable) >> 32 into the
    burnable cells in row-major order -- exact integer arithmetic on the
    known-answer-pinned Philox block."""
    rng = np.random.default_rng(9)
    fuel = rng.integers(0, 3, (23, 37)).astype(np.uint8)
    unb = (rng.random((23, 37)) < 0.1).astype(np.uint8)
    burnable = np.flatnonzero(((fuel != 0) & (unb == 0)).ravel())
    for seed in (1, 1002, 2 ** 40 + 17):
        o = oracle.Oracle(fuel, unburnable=unb, weather=S.constant_weather(1), hours=1,
                          ignition_mode=1, seed=seed, n_replicas=64)
        for r in range(64):
            x = oracle.philox4x32_10([r, 0, 0, 1], [seed & 0xFFFFFFFF, seed >> 32])
            assert o.ignition_cell(r) == burnable[(x[0] * len(burnable)) >> 32]
        o.close()


def test_burning_hours_and_scenario_draws_equal_their_integer_mappings():
    """The per-replica draws of the burning-hours limit (counter (replica, 0, 0,
    3): B = min + (x0 (max - min + 1)) >> 32) and of the weather scenario
    (counter (replica, 0, 0, 2): the first s with x0 < T_s, T_s = floor(2^32
    cum_s / total), T_last = 2^32) against exact integer arithmetic on the
    known-answer-pinned Philox blocks."""
    fuel = np.ones((5, 5), np.uint8)
    probs = [1.0, 2.0, 3.0, 4.0, 0.0, 5.0]
    total = sum(probs)
    cum = np.cumsum(probs)
    thr = [int((c / total) * 2.0 ** 32) for c in cum[:-1]] + [2 ** 32]
    assert list(oracle.scenario_thresholds(probs)) == thr
    for seed in (3, 2 ** 35 + 1):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        o = oracle.Oracle(fuel, weather=S.constant_weather(1), hours=1, seed=seed,
                          burn_hours_min=3, burn_hours_max=17)
        for r in range(200):
            x = oracle.philox4x32_10([r, 0, 0, 3], key)
            assert o.burn_hours(r) == 3 + ((x[0] * 15) >> 32)
            x = oracle.philox4x32_10([r, 0, 0, 2], key)
            want = next(s for s, t in enumerate(thr) if x[0] < t)
            assert oracle.scenario_of(seed, r, thr) == want
        o.close()
