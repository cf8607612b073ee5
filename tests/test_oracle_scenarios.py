"""Oracle pins: weather scenarios (Sec. 3.1, uncertainty source (3)).

A request may carry several weather streams with probabilities; each replica
runs under one of them.  The draw: x0 = first word of the replica's Philox
block at counter (replica, 0, 0, 2); the replica takes the first s with
x0 < T_s, T_s = floor(2^32 cum_s / total), T_{S-1} = 2^32.  Pinned by the
thresholds' closed forms, the strict-inequality boundary (brute force with
the known-answer-pinned generator), the sampled frequencies against the
probabilities, and runs that must reduce to single-weather runs.
"""
import math

import numpy as np
import pytest

import c2f_synth as S
import oracle

TWO32 = 1 << 32


def test_thresholds_closed_forms():
    assert list(oracle.scenario_thresholds([1, 1, 2])) == [TWO32 // 4, TWO32 // 2, TWO32]
    assert list(oracle.scenario_thresholds([0.25, 0.25, 0.5])) == [TWO32 // 4, TWO32 // 2, TWO32]
    assert list(oracle.scenario_thresholds([5.0])) == [TWO32]
    assert list(oracle.scenario_thresholds([0, 1])) == [0, TWO32]
    assert list(oracle.scenario_thresholds([1, 0])) == [TWO32, TWO32]
    # 1/3 of 2^32 is not an integer: floor
    assert list(oracle.scenario_thresholds([1, 1, 1])) == [TWO32 // 3, (2 * TWO32) // 3, TWO32]


@pytest.mark.parametrize("bad", [[], [-1.0, 2.0], [0.0, 0.0], [float("nan"), 1.0],
                                 [float("inf"), 1.0]])
def test_thresholds_reject_bad_probabilities(bad):
    with pytest.raises(ValueError):
        oracle.scenario_thresholds(bad)


def test_single_scenario_is_always_zero():
    t = oracle.scenario_thresholds([0.7])
    assert all(oracle.scenario_of(3, r, t) == 0 for r in range(200))


def test_strict_inequality_at_the_threshold():
    """x0 equal to T_0 goes to scenario 1; x0 one below goes to 0."""
    seed = 0x1234_5678_9ABC
    for r in (0, 1, 77, 4095):
        x0 = oracle.philox4x32_10([r, 0, 0, 2], [seed & 0xFFFFFFFF, seed >> 32])[0]
        assert oracle.scenario_of(seed, r, np.array([x0, TWO32], dtype=np.uint64)) == 1
        assert oracle.scenario_of(seed, r, np.array([x0 + 1, TWO32], dtype=np.uint64)) == 0
        # a zero-width scenario in between is skipped
        t = np.array([x0, x0, x0 + 1, TWO32], dtype=np.uint64)
        assert oracle.scenario_of(seed, r, t) == 2


def test_frequencies_follow_the_probabilities():
    probs = np.array([0.1, 0.0, 0.3, 0.6, 0.0])
    t = oracle.scenario_thresholds(probs)
    n = 40000
    got = np.bincount([oracle.scenario_of(11, r, t) for r in range(n)], minlength=5)
    assert got[1] == 0 and got[4] == 0
    for s in (0, 2, 3):
        p = probs[s] / probs.sum()
        sd = math.sqrt(n * p * (1 - p))
        assert abs(got[s] - n * p) < 5 * sd, (s, got[s], n * p)


def test_draw_does_not_reuse_the_ignition_block():
    """The scenario and the ignition cell come from different blocks: with two
    equiprobable scenarios, the scenario is not a function of the ignition
    draw's parity (it would be if both read counter (r, 0, 0, 1))."""
    t = oracle.scenario_thresholds([1, 1])
    seed = 5
    agree = 0
    for r in range(4000):
        x_ign = oracle.philox4x32_10([r, 0, 0, 1], [seed, 0])[0]
        agree += (oracle.scenario_of(seed, r, t) == (1 if x_ign >= TWO32 // 2 else 0))
    assert 1800 < agree < 2200


def _world(side=36, hours=3, seed=21):
    w = S.config2(side=side, n_replicas=6, hours=hours)
    w.params["seed"] = seed
    w.params["ros_sigma"] = 0.2
    wa = w.weather
    wb = S.weather_stream(hours, seed=seed + 1000)
    return w, wa, wb


def test_one_hot_probabilities_reduce_to_that_weather():
    w, wa, wb = _world()
    L = w.landscape
    so = oracle.ScenarioOracle(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size,
                               weathers=[wa, wb], probs=[0.0, 1.0], **w.params)
    ob = oracle.Oracle(L.fuel, L.slope, L.aspect, L.unburnable, cell_size=L.cell_size,
                       weather=wb, **w.params)
    for r in range(6):
        a, b = so.run_replica(r), ob.run_replica(r)
        assert a["scenario"] == 1
        assert np.array_equal(a["ign"], b["ign"]) and a["work"] == b["work"]
        assert a["ignition_cell"] == b["ignition_cell"]


def test_identical_scenarios_reduce_to_one_weather():
    w, wa, _ = _world(seed=22)
    L = w.landscape
    so = oracle.ScenarioOracle(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size,
                               weathers=[wa, wa, wa], probs=[1, 2, 3], **w.params)
    o = oracle.Oracle(L.fuel, L.slope, L.aspect, L.unburnable, cell_size=L.cell_size,
                      weather=wa, **w.params)
    seen = set()
    for r in range(6):
        a, b = so.run_replica(r), o.run_replica(r)
        seen.add(a["scenario"])
        assert np.array_equal(a["ign"], b["ign"]) and a["work"] == b["work"]
    assert len(seen) > 1


def test_scenarios_change_the_fire():
    """Two different weather streams: some replica's scar depends on which one
    it drew (the table rows of the two scenarios differ)."""
    w, wa, wb = _world(seed=23)
    L = w.landscape
    so = oracle.ScenarioOracle(L.fuel, L.slope, L.aspect, L.unburnable, L.cell_size,
                               weathers=[wa, wb], probs=[1, 1], **w.params)
    cell = int(np.flatnonzero(L.fuel.ravel())[0])
    assert not np.array_equal(so.base_inc(0, cell, 0)[0], so.base_inc(1, cell, 0)[0])
    oa = oracle.Oracle(L.fuel, L.slope, L.aspect, L.unburnable, cell_size=L.cell_size,
                       weather=wa, **w.params)
    ob = oracle.Oracle(L.fuel, L.slope, L.aspect, L.unburnable, cell_size=L.cell_size,
                       weather=wb, **w.params)
    differs = False
    for r in range(6):
        ra, rb = oa.run_replica(r), ob.run_replica(r)
        differs |= not np.array_equal(ra["ign"], rb["ign"])
        got = so.run_replica(r)
        ref = ra if got["scenario"] == 0 else rb
        assert np.array_equal(got["ign"], ref["ign"])
    assert differs
