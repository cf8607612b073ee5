"""Oracle pins: burning hours per day (A5, general fire dynamics condition (1)).

A replica's fire burns only in the first B hours of each day of the weather
stream (h mod 24 < B); in the other hours it is dormant.  B is a constant or
drawn per replica uniformly from {min..max} (Philox counter (replica, 0, 0, 3)).
Pinned by: B = 24 equals no limit; with no perturbation, a run with dormant
hours equals the unlimited run on the stream of its burning hours alone (same
scar and work, ignition steps shifted by the dormant periods before them);
the draw's range and frequencies; and the event search (O2), a different
algorithm over ignition steps, equal to the stepped loop (O1) with the limit.
"""
import math

import numpy as np
import pytest

import c2f_synth as S
import oracle


def _mk(w, weather=None, **over):
    L = w.landscape
    return oracle.Oracle(L.fuel, L.slope, L.aspect, L.unburnable, cell_size=L.cell_size,
                         weather=w.weather if weather is None else weather, **dict(w.params, **over))


def _world(hours=30, seed=7, side=34):
    w = S.config2(side=side, n_replicas=4, hours=hours)
    w.weather = S.weather_stream(hours, seed=seed, ws_mean=12.0)
    w.params["seed"] = seed
    return w


def test_24_hours_is_no_limit():
    w = _world()
    a, b = _mk(w), _mk(w, burn_hours_min=24, burn_hours_max=24)
    for r in range(4):
        ra, rb = a.run_replica(r), b.run_replica(r)
        assert np.array_equal(ra["ign"], rb["ign"]) and ra["work"] == rb["work"]


@pytest.mark.parametrize("B,mps", [(5, 1), (1, 1), (3, 10)])
def test_dormant_hours_equal_the_stream_of_burning_hours(B, mps):
    """sigma = 0: the fire with dormant hours is the unlimited fire on the
    weather of its burning hours only, hours renumbered."""
    H = 52
    w = _world(hours=H, seed=11)
    w.params.update(ros_sigma=0.0, minutes_per_step=mps)
    active = [h for h in range(H) if h % 24 < B]
    lim = _mk(w, burn_hours_min=B, burn_hours_max=B)
    comp = _mk(w, weather=np.asarray(w.weather)[active], hours=len(active))
    sph = 60 // mps
    for r in range(4):
        assert lim.burn_hours(r) == B
        rl, rc = lim.run_replica(r), comp.run_replica(r)
        assert np.array_equal(rl["scar"], rc["scar"]), r
        assert rl["work"] == rc["work"] and rl["n_ignited"] == rc["n_ignited"], r
        # step s of burning hour active[k] is step s - (active[k] - k) sph of the compressed run
        il = rl["ign"].ravel()
        shifted = il.copy()
        pos = il > 0
        hour = (il[pos] - 1) // sph
        k = np.searchsorted(active, hour)
        assert np.array_equal(np.asarray(active)[k], hour)   # ignitions only in burning hours
        shifted[pos] = il[pos] - (hour - k) * sph
        assert np.array_equal(shifted, rc["ign"].ravel()), r


def test_draw_range_and_frequencies():
    w = _world(hours=2)
    o = _mk(w, burn_hours_min=3, burn_hours_max=8)
    n = 24000
    got = np.array([o.burn_hours(r) for r in range(n)])
    assert got.min() == 3 and got.max() == 8
    counts = np.bincount(got - 3, minlength=6)
    p = 1 / 6
    sd = math.sqrt(n * p * (1 - p))
    assert (np.abs(counts - n * p) < 5 * sd).all(), counts
    # the draw is the published generator's first word at counter (r, 0, 0, 3)
    for r in (0, 5, 999):
        x0 = oracle.philox4x32_10([r, 0, 0, 3], [w.params["seed"] & 0xFFFFFFFF, w.params["seed"] >> 32])[0]
        assert o.burn_hours(r) == 3 + (x0 * 6 >> 32)


def test_no_limit_reports_24():
    w = _world(hours=2)
    assert _mk(w).burn_hours(0) == 24


@pytest.mark.parametrize("seed", range(6))
def test_event_search_equals_stepped_loop_with_dormant_hours(seed):
    """O2 = O1 under a burning-hours limit: noise, drawn B in {2..9}, a delta
    burn-out or a threshold on alternate seeds, 1- and 5-minute clocks."""
    w = _world(hours=50, seed=seed)
    over = dict(burn_hours_min=2, burn_hours_max=9, ros_sigma=0.3,
                minutes_per_step=5 if seed % 3 == 2 else 1)
    if seed % 2:
        over["burnout_delta"] = 1.0
    else:
        over["ros_threshold"] = 0.5
    o = _mk(w, **over)
    for r in range(4):
        a, b = o.run_replica(r), o.run_replica_event(r)
        assert np.array_equal(a["ign"], b["ign"]), r
        assert a["work"] == b["work"] and a["n_ignited"] == b["n_ignited"], r
