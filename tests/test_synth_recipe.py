"""The synthetic inputs follow their stated recipe (no GPU).

The benchmark workloads stand in for the paper's unavailable instances, so
their value distributions are part of the claim: these checks tie the seeded
generators to the recipe (10 % non-fuel, the heterogeneous fuel set, slopes
scaled to a 99th percentile of 40 %, downslope aspects, hourly weather in the
stated ranges, the batch and request-stream size distributions).
"""
import math

import numpy as np

import c2f_synth as S


def test_headline_landscape_recipe():
    L = S.config2().landscape
    assert L.fuel.shape == (512, 512) and L.fuel.dtype == np.uint8 and L.cell_size == 100.0
    assert abs((L.fuel == 0).mean() - 0.10) < 0.002                 # the non-fuel fraction
    codes = {S.FUEL_CODES[f] for f in S.HETERO_FUELS}
    present = set(np.unique(L.fuel).tolist()) - {0}
    assert present == codes                                          # every fuel of the set, no other
    shares = np.array([(L.fuel == c).mean() for c in sorted(codes)]) / 0.9
    assert shares.min() > 0.05 and shares.max() < 0.15               # clustered, but none dominant
    assert L.slope.dtype == np.float32 and L.slope.min() >= 0.0 and L.slope.max() <= 40.0
    assert abs(np.quantile(L.slope, 0.99) - 40.0) < 0.05             # scaled to p99 = 40 %, clipped
    assert L.aspect.min() >= 0.0 and L.aspect.max() < 360.0
    # clustered fuel: neighbouring cells mostly share a fuel (8x8-cell lattice noise)
    same = (L.fuel[:, 1:] == L.fuel[:, :-1]).mean()
    assert same > 0.8


def test_weather_stream_recipe():
    w = S.weather_stream(24 * 400, seed=7)
    ws, wd, ffmc, bui = w.T
    assert w.shape == (9600, 4) and w.dtype == np.float64
    assert abs(ws.mean() - 20.0) < 0.3 and abs(ws.std() - 5.0) < 0.3 and ws.min() >= 0.0
    assert wd.min() >= 0.0 and wd.max() < 360.0
    steps = (np.diff(wd) + 180.0) % 360.0 - 180.0                    # the direction's random walk
    assert abs(steps.std() - 15.0) < 0.5 and wd[0] == 270.0
    assert ffmc.min() >= 85.0 and ffmc.max() <= 93.0
    assert np.all(bui == bui[0]) and 40.0 <= bui[0] <= 120.0          # one BUI per stream
    shifted = S.weather_stream(72, seed=7, shift_at=36)
    plain = S.weather_stream(72, seed=7)
    d = (shifted[:, 1] - plain[:, 1]) % 360.0
    assert np.all(d[:36] == 0.0) and np.allclose(d[36:], 90.0)       # the +90 degree shift at hour 36


def test_batch_and_request_stream_recipes():
    specs = S.config3_specs()
    sides = np.array([s["side"] for s in specs])
    reps = np.array([s["n_replicas"] for s in specs])
    assert len(specs) == 64 and sides.min() >= 64 and sides.max() <= 2048
    assert reps.min() >= 16 and reps.max() <= 4096 and all(s["hours"] == 48 for s in specs)
    assert int((sides ** 2).sum()) == 37882754 and int(reps.sum()) == 41489
    # log-uniform: the log sides spread like a uniform over [ln 64, ln 2048] (std = range / sqrt 12)
    assert np.log(sides).std() > 0.75 * (math.log(2048) - math.log(64)) / math.sqrt(12)
    pool, reqs = S.serving_requests(rate=50.0, duration_s=60.0)
    assert len(pool) == 16 and min(pool) >= 128 and max(pool) <= 2048
    t = np.array([r["arrival_s"] for r in reqs])
    assert abs(len(reqs) / 60.0 - 50.0) < 3.0                        # Poisson arrivals at 50/s
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 0.02) < 0.002 and abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    rr = np.array([r["n_replicas"] for r in reqs])
    hh = np.array([r["hours"] for r in reqs])
    assert rr.min() >= 32 and rr.max() <= 2048 and hh.min() >= 12 and hh.max() <= 72


def test_scenario_set_recipe():
    weathers, weights = S.scenario_set(8, 24)
    assert weathers.shape == (8, 24, 4) and list(weights) == [1, 2, 3, 4, 4, 3, 2, 1]
    means = weathers[:, :, 0].mean(axis=1)
    assert np.all(np.diff(means) > 0)                                # calm to strong wind
    assert [float(weathers[s, 0, 1]) for s in range(8)] == [(270.0 + 20.0 * s) % 360.0 for s in range(8)]
