"""Pins of the oracle's step loop (Algorithm 1) and burn-probability count.

- hand-enumerated ignition steps and work counts on 3x3 and 5x5 grids
  (tests/golden, derived by hand from Secs. 3.1, 3.3, 3.4 and A5);
- arrival time ceil(d / ROS) along rows;
- exact symmetries: circle under the 8 symmetries of the square, rotating
  and mirroring the wind rotates and mirrors the scar;
- brute force: the label-setting search (O2) equals the stepped loop (O1)
  on random small landscapes, including noise, thresholds and delta burn-out;
- the threshold and delta rules of Sec. 3.1 and A5 (i).
"""
import numpy as np
import pytest

import c2f_synth as S
import oracle
from conftest import read_golden_grid


def homog(rows, cols, wd=270.0, ws=0.0, hours=1, unburnable=None, **params):
    fuel = np.full((rows, cols), 1, dtype=np.uint8)
    weather = S.constant_weather(hours, ws=ws, wd_from=wd)
    p = dict(hours=hours, ignition_mode=0, ignition_cell=(rows // 2) * cols + cols // 2)
    p.update(params)
    return oracle.Oracle(fuel, unburnable=unburnable, weather=weather, **p)


def harvested_mask(meta, shape):
    """The golden's harvested cells (key harvested_col: one whole column), or None."""
    if "harvested_col" not in meta:
        return None
    unb = np.zeros(shape, np.uint8)
    unb[:, int(meta["harvested_col"])] = 1
    return unb


@pytest.mark.parametrize("name", ["hand_3x3.txt", "hand_5x5.txt", "hand_wind_eq1_5x5.txt",
                                  "hand_wind_ray_5x5.txt", "hand_delta_5x5.txt",
                                  "hand_threshold_5x5.txt", "hand_burnhours_3x3.txt",
                                  "hand_clock5_3x3.txt", "hand_harvested_5x5.txt"])
@pytest.mark.parametrize("runner", ["run_replica", "run_replica_event"])
def test_hand_enumeration(name, runner):
    """Hand-enumerated ignition steps and work: constant rates on all axes, and
    under wind the ellipse of chosen (H, B, LB) by Eq. (1) and by the ray of
    ellipse_mode 1, each axis's rate derived by hand; burn-out below delta
    (A5 (i)), rejected messages under a receive threshold, a fire that burns
    one hour a day (A5, condition (1)), a 5-minute clock and a harvested
    column (tests/golden/)."""
    meta, grid = read_golden_grid(name)
    g = np.array(grid)
    bh = (int(meta.get("burn_hours_min", 0)), int(meta.get("burn_hours_max", 0)))
    o = homog(g.shape[0], g.shape[1], hours=int(meta["hours"]), const_ros=float(meta["const_ros"]),
              unburnable=harvested_mask(meta, g.shape),
              wd=float(meta.get("wd_from", 270.0)), ws=float(meta.get("ws", 0.0)),
              const_bros=float(meta.get("const_bros", 0.0)), const_lb=float(meta.get("const_lb", 0.0)),
              ellipse_mode=int(meta.get("ellipse_mode", 0)),
              burnout_delta=float(meta.get("burnout_delta", 0.0)),
              ros_threshold=float(meta.get("ros_threshold", 0.0)),
              burn_hours_min=bh[0], burn_hours_max=bh[1],
              minutes_per_step=int(meta.get("minutes_per_step", 1)))
    r = getattr(o, runner)(0)
    assert np.array_equal(r["ign"], g)
    assert r["work"] == int(meta["work"])
    assert r["n_ignited"] == int((g >= 0).sum())


def test_arrival_time_is_distance_over_rate():
    # 1 x 41 strip, constant ROS: cell at distance d ignites at ceil(100 d / ros) per hop
    for ros in (7.0, 10.0, 33.0, 99.0):
        o = homog(1, 41, hours=3, const_ros=ros)
        r = o.run_replica(0)
        hop = int(np.ceil(100.0 / ros))
        ign = r["ign"][0]
        for d in range(0, 21):
            expect = d * hop if d * hop <= o.steps else -1
            assert ign[20 + d] == expect and ign[20 - d] == expect


def test_circle_is_invariant_under_square_symmetries():
    o = homog(31, 31, ws=0.0, hours=4)
    ign = o.run_replica(0)["ign"]
    for k in range(4):
        assert np.array_equal(np.rot90(ign, k), ign)
        assert np.array_equal(np.fliplr(np.rot90(ign, k)), ign)


def test_rotating_the_wind_rotates_the_scar():
    east = homog(41, 41, wd=270.0, ws=25.0, hours=3).run_replica(0)["ign"]
    north = homog(41, 41, wd=180.0, ws=25.0, hours=3).run_replica(0)["ign"]
    west = homog(41, 41, wd=90.0, ws=25.0, hours=3).run_replica(0)["ign"]
    assert np.array_equal(np.rot90(east), north)
    assert np.array_equal(np.fliplr(east), west)
    assert (east[:, 21:] >= 0).sum() > (east[:, :20] >= 0).sum()   # grows downwind


@pytest.mark.parametrize("seed", range(24))
def test_event_search_equals_stepped_loop(seed):
    w = S.random_small_case(seed)
    L = w.landscape
    o = oracle.Oracle(L.fuel, L.slope, L.aspect, L.unburnable, weather=w.weather, **w.params)
    if o.lib.or_ignition_cell(o._h, 0) < 0:
        pytest.skip("no burnable cell")
    for r in range(3):
        a, b = o.run_replica(r), o.run_replica_event(r)
        assert np.array_equal(a["ign"], b["ign"])
        assert a["work"] == b["work"] and a["n_ignited"] == b["n_ignited"]


def test_event_search_equals_stepped_loop_on_workload_sample():
    w = S.config2(side=96, n_replicas=4, hours=6)
    L = w.landscape
    o = oracle.Oracle(L.fuel, L.slope, L.aspect, weather=w.weather, **w.params)
    for r in range(4):
        a, b = o.run_replica(r), o.run_replica_event(r)
        assert np.array_equal(a["ign"], b["ign"]) and a["work"] == b["work"]


def test_threshold_blocks_ignition():
    o = homog(5, 5, const_ros=10.0, ros_threshold=10.0)   # needs ROS > 10
    r = o.run_replica(0)
    assert r["n_ignited"] == 1 and r["work"] == o.steps    # the centre keeps burning
    o = homog(5, 5, const_ros=10.0, ros_threshold=9.99)
    assert o.run_replica(0)["n_ignited"] == 25


def test_delta_burnout():
    o = homog(5, 5, const_ros=10.0, burnout_delta=20.0)
    r = o.run_replica(0)
    assert r["n_ignited"] == 1 and r["work"] == 1        # sends in step 1, burned after it


def test_isolated_ignition_burns_out_after_one_step():
    fuel = np.zeros((3, 3), dtype=np.uint8); fuel[1, 1] = 1
    o = oracle.Oracle(fuel, weather=S.constant_weather(1), hours=1, ignition_cell=4)
    r = o.run_replica(0)
    assert r["work"] == 1 and r["n_ignited"] == 1


def test_uniform_ignition_hits_only_burnable_cells():
    w = S.config2(side=64, n_replicas=1, hours=1)
    L = w.landscape
    o = oracle.Oracle(L.fuel, L.slope, L.aspect, weather=w.weather, **w.params)
    cells = [o.ignition_cell(r) for r in range(400)]
    assert all(L.fuel.ravel()[c] != 0 for c in cells)
    assert len(set(cells)) > 300


def test_burn_prob_counts():
    w = S.config2(side=64, n_replicas=6, hours=3)
    L = w.landscape
    o = oracle.Oracle(L.fuel, L.slope, L.aspect, weather=w.weather, **w.params)
    scars = np.stack([o.run_replica(r)["scar"] for r in range(6)])
    bp = oracle.burn_prob(scars)
    assert bp.dtype == np.uint32 and bp.max() <= 6
    assert np.array_equal(bp, scars.sum(0))
    assert np.array_equal(oracle.burn_prob(scars[:1]), scars[0])


def test_smaller_steps_change_the_scar_little():
    """Sec. 3.1: a finer clock barely changes the final scar (sanity, not parity)."""
    w = S.config1()
    L = w.landscape
    a = oracle.Oracle(L.fuel, weather=w.weather, **dict(w.params, minutes_per_step=1)).run_replica(0)
    b = oracle.Oracle(L.fuel, weather=w.weather, **dict(w.params, minutes_per_step=2)).run_replica(0)
    diff = (a["scar"] != b["scar"]).sum()
    assert diff <= 0.1 * a["scar"].sum()


def _strip_by_integers(seed, sigma, ros, n, hours, thr=0.0, burn_hours=24):
    """Ignition steps and work of a 1 x n strip (centre ignition, constant rate
    `ros` on every axis, 1-minute clock) by exact integer arithmetic: per step s
    (weather hour (s - 1) // 60) a burning cell i advances by
    inc = min((B F + 2^31) >> 32, D), B = ros 2^32, F = f 2^32 with f the
    perturbation of (replica 0, i, hour), D = 100 m in 2^-32 m units; its
    neighbour is reached at the first step where the sum of its increments since
    it ignited reaches D, and ignites if ros f > thr (binary64 product, its own
    perturbation at that hour; a rejected message is consumed, so a strip's
    fire stops there); a cell burns until its last neighbour has ignited.  With
    burn_hours B < 24 the steps of weather hours h with h mod 24 >= B are dormant:
    no progress and no work (A5, condition (1))."""
    D = 100 * 2 ** 32
    B = int(round(ros * 2 ** 32))
    steps = 60 * hours
    incs = {}

    def inc(i, h):
        if (i, h) not in incs:
            f = float(oracle.noise_factor(seed, 0, i, h, sigma))
            F = int(f * 2 ** 32)
            assert F == f * 2 ** 32                              # f 2^32 is an integer
            incs[i, h] = min((B * F + 2 ** 31) >> 32, D)
        return incs[i, h]

    c = n // 2
    ign = [-1] * n
    ign[c] = 0
    for d in (1, -1):
        i = c
        while 0 <= i + d < n:
            p, s = 0, ign[i]
            while p < D and s < steps:
                s += 1
                if ((s - 1) // 60) % 24 < burn_hours:
                    p += inc(i, (s - 1) // 60)
            if p < D:
                break
            f_next = float(oracle.noise_factor(seed, 0, i + d, (s - 1) // 60, sigma))
            if not ros * f_next > thr:
                break
            ign[i + d] = s
            i += d
    def burning_steps(a, b):         # steps a+1..b outside dormant hours
        return sum(1 for s in range(a + 1, b + 1) if ((s - 1) // 60) % 24 < burn_hours)

    work = 0
    for i in range(n):
        if ign[i] >= 0:
            nb = [ign[j] for j in (i - 1, i + 1) if 0 <= j < n]
            work += burning_steps(ign[i], max(nb) if min(nb) >= 0 else steps)
    return np.array(ign), work


@pytest.mark.parametrize("seed,sigma", [(1, 0.1), (7, 0.5), (12345, 1.0)])
@pytest.mark.parametrize("runner", ["run_replica", "run_replica_event"])
def test_noisy_strip_equals_its_integer_model(seed, sigma, runner):
    """[R2] with the perturbation applied in integers, and progress carried across
    weather hours (Alg. 1): a noisy 3-hour strip against exact big-integer
    arithmetic on the perturbations (pinned against a float64 Box-Muller in
    test_oracle_math.py)."""
    n, hours = 101, 3
    fuel = np.ones((1, n), np.uint8)
    o = oracle.Oracle(fuel, weather=S.constant_weather(hours, ws=0.0), hours=hours, ignition_mode=0,
                      ignition_cell=n // 2, const_ros=30.0, ros_sigma=sigma, seed=seed)
    ign, work = _strip_by_integers(seed, sigma, 30.0, n, hours)
    r = getattr(o, runner)(0)
    assert np.array_equal(r["ign"][0], ign)
    assert r["work"] == work
    assert (ign > 60).any()                                      # crossings after the first hour


@pytest.mark.parametrize("seed", [11, 21, 42])
def test_noisy_strip_with_a_receive_threshold(seed):
    """Sec. 3.1 receive test with noise: a messaged cell ignites only if
    HROS f > threshold; here HROS = 30 m/min and the threshold 25 m/min, so a
    cell whose perturbation is below 5/6 rejects its message and stops the
    strip's fire on that side; the integer model decides each test in binary64
    like the oracle."""
    n, hours = 101, 3
    fuel = np.ones((1, n), np.uint8)
    o = oracle.Oracle(fuel, weather=S.constant_weather(hours, ws=0.0), hours=hours, ignition_mode=0,
                      ignition_cell=n // 2, const_ros=30.0, ros_sigma=0.2, seed=seed, ros_threshold=25.0)
    ign, work = _strip_by_integers(seed, 0.2, 30.0, n, hours, thr=25.0)
    free, _ = _strip_by_integers(seed, 0.2, 30.0, n, hours)
    r = o.run_replica(0)
    assert np.array_equal(r["ign"][0], ign) and r["work"] == work
    assert 1 < (ign >= 0).sum() < (free >= 0).sum()              # accepted, then rejected messages


def _strip_with_delta(seed, sigma, ros, n, hours, delta):
    """A 1 x n noisy strip under the delta burn-out of A5 (i), by exact integer
    arithmetic: a cell whose ros f is below delta in the hour it ignites is
    Burned at the end of its ignition period and sends nothing; a burning cell
    whose ros f falls below delta at a later hour boundary (the ignition cell:
    at hour 0) still advances in that hour's first period and is Burned after
    it; otherwise as _strip_by_integers, and a cell also burns out once its last
    neighbour has ignited (A5 (ii))."""
    D = 100 * 2 ** 32
    B = int(round(ros * 2 ** 32))
    steps = 60 * hours

    def f(i, h):
        return float(oracle.noise_factor(seed, 0, i, h, sigma))

    def inc(i, h):
        return min((B * int(f(i, h) * 2 ** 32) + 2 ** 31) >> 32, D)

    def dies(i, h):
        return ros * f(i, h) < delta

    def timeline(i, t):
        """(step at which cell i, ignited at t, reaches its outward neighbour or
        None, step at whose end A5 (i) burns it or None)."""
        h_t = (t - 1) // 60 if t >= 1 else 0
        if t >= 1 and dies(i, h_t):
            return None, t
        p, cross = 0, None
        for s in range(t + 1, steps + 1):
            h = (s - 1) // 60
            boundary = s == 60 * h + 1 and (t == 0 or h > h_t)
            if cross is None:
                p += inc(i, h)
                if p >= D:
                    cross = s
            if boundary and dies(i, h):
                return cross, s
        return cross, None

    c = n // 2
    ign = [-1] * n
    ign[c] = 0
    for d in (1, -1):
        i = c
        while 0 <= i + d < n:
            cross, _ = timeline(i, ign[i])
            if cross is None:
                break
            ign[i + d] = cross
            i += d
    work = 0
    for i in range(n):
        if ign[i] < 0:
            continue
        nb = [ign[j] for j in (i - 1, i + 1) if 0 <= j < n]
        ends = [x for x in (timeline(i, ign[i])[1], max(nb) if min(nb) >= 0 else None) if x is not None]
        work += (min(ends) if ends else steps) - ign[i]
    return np.array(ign), work


@pytest.mark.parametrize("seed", [2, 5, 13])
def test_noisy_strip_with_delta_burnout(seed):
    """A5 (i) with noise over 4 hours: cells die when their perturbed HROS is
    below delta = 22 m/min (HROS 30, sigma 0.2), at ignition or at a later hour
    boundary; ignition steps and work against the integer model."""
    n, hours = 201, 4
    fuel = np.ones((1, n), np.uint8)
    o = oracle.Oracle(fuel, weather=S.constant_weather(hours, ws=0.0), hours=hours, ignition_mode=0,
                      ignition_cell=n // 2, const_ros=30.0, ros_sigma=0.2, seed=seed, burnout_delta=22.0)
    ign, work = _strip_with_delta(seed, 0.2, 30.0, n, hours, 22.0)
    r = o.run_replica(0)
    assert np.array_equal(r["ign"][0], ign) and r["work"] == work
    assert (ign >= 0).sum() > 5                                  # the fire runs, then dies out


@pytest.mark.parametrize("seed", [4, 9])
@pytest.mark.parametrize("runner", ["run_replica", "run_replica_event"])
def test_noisy_strip_burning_three_hours_a_day(seed, runner):
    """A5 condition (1) with noise: over 30 hours a fire that burns only the first
    3 hours of each day (hours 0-2 and 24-26) against the integer model with the
    other hours dormant; the stepped loop (O1) and the event search (O2)."""
    n, hours = 201, 30
    fuel = np.ones((1, n), np.uint8)
    o = oracle.Oracle(fuel, weather=S.constant_weather(hours, ws=0.0), hours=hours, ignition_mode=0,
                      ignition_cell=n // 2, const_ros=30.0, ros_sigma=0.3, seed=seed,
                      burn_hours_min=3, burn_hours_max=3)
    ign, work = _strip_by_integers(seed, 0.3, 30.0, n, hours, burn_hours=3)
    r = getattr(o, runner)(0)
    assert np.array_equal(r["ign"][0], ign) and r["work"] == work
    assert (ign > 24 * 60).any()                                 # it burns again on the second day
