"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's instances (Dogrib, the BurnP3 British Columbia landscapes, the
Yaha Tinda weather) are not available, so these generators stand in for
them: 100 m cells, FBP fuel codes, slope/aspect from a synthetic elevation
model and hourly weather streams (Sec. 3.5 inputs; Sec. 4.2 and App. A
instance sizes).  This module holds no part of the fire-growth method: it
only draws inputs, and both the GPU library and the CPU oracle consume them.

Fuel grid codes (uint8): 0 non-fuel, 1 C1, 2 C2, 3 C3, 4 C4, 5 C5, 6 C6,
7 C7, 8 D1, 9 M1, 10 M2, 11 O1a, 12 O1b, 13 S1, 14 S2, 15 S3.
Weather rows: (ws_kmh, wd_from_deg, ffmc, bui).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FUEL_CODES = {"C1": 1, "C2": 2, "C3": 3, "C4": 4, "C5": 5, "C6": 6, "C7": 7, "D1": 8,
              "M1": 9, "M2": 10, "O1a": 11, "O1b": 12, "S1": 13, "S2": 14, "S3": 15}
HETERO_FUELS = ("C1", "C2", "C3", "C4", "C6", "C7", "D1", "M1", "O1a", "S1")


@dataclass
class Landscape:
    fuel: np.ndarray                      # uint8 (rows, cols)
    slope: np.ndarray                     # float32 percent
    aspect: np.ndarray                    # float32 degrees, downslope azimuth clockwise from N
    cell_size: float = 100.0
    unburnable: np.ndarray | None = None  # uint8, 1 = harvested

    @property
    def shape(self):
        return self.fuel.shape


@dataclass
class Workload:
    landscape: Landscape
    weather: np.ndarray                   # float64 (hours, 4)
    params: dict = field(default_factory=dict)


def _value_noise(rng, rows, cols, period, n_fields=1):
    """Bilinearly interpolated lattice noise with the given lattice period (cells)."""
    ny = int(math.ceil(rows / period)) + 1
    nx = int(math.ceil(cols / period)) + 1
    lat = rng.random((n_fields, ny, nx))
    y = (np.arange(rows) + 0.5) / period
    x = (np.arange(cols) + 0.5) / period
    y0 = np.floor(y).astype(np.int64); x0 = np.floor(x).astype(np.int64)
    fy = (y - y0)[:, None]; fx = (x - x0)[None, :]
    out = np.empty((n_fields, rows, cols), dtype=np.float64)
    for f in range(n_fields):
        v = lat[f]
        a = v[y0][:, x0]; b = v[y0][:, x0 + 1]
        c = v[y0 + 1][:, x0]; d = v[y0 + 1][:, x0 + 1]
        out[f] = (a * (1 - fx) + b * fx) * (1 - fy) + (c * (1 - fx) + d * fx) * fy
    return out


def _fbm(rng, rows, cols, octaves=6, base_period=256, gain=0.5):
    z = np.zeros((rows, cols), dtype=np.float64)
    amp = 1.0
    for o in range(octaves):
        period = max(base_period / (2 ** o), 1.0)
        z += amp * _value_noise(rng, rows, cols, period)[0]
        amp *= gain
    return z


def _horn(z, cell_size):
    """Horn's 3x3 slope (percent) and downslope aspect (deg clockwise from N), edges replicated."""
    p = np.pad(z, 1, mode="edge")
    a = p[:-2, :-2]; b = p[:-2, 1:-1]; c = p[:-2, 2:]
    d = p[1:-1, :-2]; f = p[1:-1, 2:]
    g = p[2:, :-2]; h = p[2:, 1:-1]; i = p[2:, 2:]
    dzdx = ((c + 2 * f + i) - (a + 2 * d + g)) / (8.0 * cell_size)   # toward east
    dzdy = ((a + 2 * b + c) - (g + 2 * h + i)) / (8.0 * cell_size)   # toward north (row 0 = north)
    slope = np.hypot(dzdx, dzdy) * 100.0
    aspect = np.degrees(np.arctan2(-dzdx, -dzdy)) % 360.0
    return slope, aspect


def heterogeneous_landscape(side_rows, side_cols=None, seed=2, cell_size=100.0,
                            fuels=HETERO_FUELS, nonfuel_frac=0.10, max_slope=40.0):
    """Clustered fuel map over `fuels` with a non-fuel fraction, fractal terrain.

    Fuel: value noise on an 8x8-cell lattice per fuel, argmax; the `nonfuel_frac`
    lowest cells of a separate field become non-fuel.  Elevation: 6-octave fBm,
    base period 256 cells, gain 0.5; slope/aspect by Horn's method, scaled so the
    99th-percentile slope is `max_slope` percent and clipped there.
    """
    rows = int(side_rows)
    cols = int(side_cols if side_cols is not None else side_rows)
    rng = np.random.default_rng(seed)
    noise = _value_noise(rng, rows, cols, 8.0, n_fields=len(fuels))
    codes = np.array([FUEL_CODES[f] for f in fuels], dtype=np.uint8)
    fuel = codes[np.argmax(noise, axis=0)]
    nf = _value_noise(rng, rows, cols, 8.0)[0]
    cut = np.quantile(nf, nonfuel_frac)
    fuel = np.where(nf <= cut, 0, fuel).astype(np.uint8)
    z = _fbm(rng, rows, cols)
    slope, aspect = _horn(z, cell_size)
    p99 = float(np.quantile(slope, 0.99))
    scale = max_slope / p99 if p99 > 0 else 0.0
    slope = np.minimum(slope * scale, max_slope)
    return Landscape(fuel=fuel, slope=slope.astype(np.float32),
                     aspect=aspect.astype(np.float32), cell_size=cell_size)


def weather_stream(hours, seed=102, ws_mean=20.0, ws_sd=5.0, wd0=270.0, wd_step_sd=15.0,
                   ffmc=(85.0, 93.0), bui=(40.0, 120.0), shift_at=None, shift_deg=90.0):
    """Hourly (ws, wd_from, ffmc, bui): normal wind speed, random-walk direction,
    uniform FFMC per hour, one uniform BUI per scenario; optional direction jump."""
    rng = np.random.default_rng(seed)
    ws = np.clip(rng.normal(ws_mean, ws_sd, hours), 0.0, None)
    steps = rng.normal(0.0, wd_step_sd, hours)
    steps[0] = 0.0
    if shift_at is not None and 0 < shift_at < hours:
        steps[shift_at] += shift_deg
    wd = (wd0 + np.cumsum(steps)) % 360.0
    ff = rng.uniform(ffmc[0], ffmc[1], hours)
    b = np.full(hours, rng.uniform(bui[0], bui[1]))
    return np.stack([ws, wd, ff, b], axis=1).astype(np.float64)


def constant_weather(hours, ws=20.0, wd_from=270.0, ffmc=90.0, bui=80.0):
    return np.tile(np.array([[ws, wd_from, ffmc, bui]], dtype=np.float64), (hours, 1))


# ------------------------------------------------------------------ configs
def config1() -> Workload:
    """40x40, 100 m, homogeneous C1, flat, constant weather (FFMC 90, BUI 80, 20 km/h
    from 270 deg), centre ignition, 10 h, 1-minute clock, deterministic, 1 replica."""
    fuel = np.full((40, 40), FUEL_CODES["C1"], dtype=np.uint8)
    z = np.zeros((40, 40), dtype=np.float32)
    land = Landscape(fuel=fuel, slope=z.copy(), aspect=z.copy())
    params = dict(seed=1, n_replicas=1, hours=10, minutes_per_step=1, ignition_mode=0,
                  ignition_cell=20 * 40 + 20, ros_sigma=0.0)
    return Workload(land, constant_weather(10), params)


def config2(side=512, n_replicas=1000, hours=24) -> Workload:
    """512x512 heterogeneous landscape, 24 h hourly weather, 1000 replicas with
    uniform random ignitions and lognormal(0, 0.1) ROS noise."""
    land = heterogeneous_landscape(side, seed=2)
    params = dict(seed=1002, n_replicas=n_replicas, hours=hours, minutes_per_step=1,
                  ignition_mode=1, ignition_cell=0, ros_sigma=0.1)
    return Workload(land, weather_stream(hours, seed=102), params)


def config3_specs(n_landscapes=64, seed=3, hours=48):
    """(side, replicas, landscape seed, weather seed) of the batching workload:
    sides log-uniform in [64, 2048], replica counts log-uniform in [16, 4096]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_landscapes):
        side = int(round(math.exp(rng.uniform(math.log(64), math.log(2048)))))
        reps = int(round(math.exp(rng.uniform(math.log(16), math.log(4096)))))
        out.append(dict(side=side, n_replicas=reps, land_seed=1000 + i, weather_seed=2000 + i,
                        run_seed=3000 + i, hours=hours))
    return out


def config3_workload(spec) -> Workload:
    land = heterogeneous_landscape(spec["side"], seed=spec["land_seed"])
    params = dict(seed=spec["run_seed"], n_replicas=spec["n_replicas"], hours=spec["hours"],
                  minutes_per_step=1, ignition_mode=1, ignition_cell=0, ros_sigma=0.1)
    return Workload(land, weather_stream(spec["hours"], seed=spec["weather_seed"]), params)


def config4(side=4096, n_replicas=256, hours=72) -> Workload:
    """4096x4096 landscape, 72 h weather with a +90 deg wind shift at hour 36, 256 replicas."""
    land = heterogeneous_landscape(side, seed=4)
    params = dict(seed=4004, n_replicas=n_replicas, hours=hours, minutes_per_step=1,
                  ignition_mode=1, ignition_cell=0, ros_sigma=0.1)
    return Workload(land, weather_stream(hours, seed=104, shift_at=36), params)


def scenario_set(n_scen=8, hours=24, seed=102):
    """Weather scenarios of one request (Sec. 3.1, uncertainty (3)): n_scen
    hourly streams, calm to strong wind (mean 8 + 4 s km/h) from directions
    20 s degrees apart, with unnormalised weights rising then falling
    (1, 2, ..., 2, 1).  Returns (weathers (n_scen, hours, 4), weights)."""
    weathers = np.stack([weather_stream(hours, seed=seed + 31 * s, ws_mean=8.0 + 4.0 * s,
                                        wd0=(270.0 + 20.0 * s) % 360.0) for s in range(n_scen)])
    half = (n_scen + 1) // 2
    w = np.concatenate([np.arange(1, half + 1), np.arange(n_scen - half, 0, -1)]).astype(np.float64)
    return weathers, w


def serving_requests(rate=50.0, duration_s=60.0, seed=5, pool=16):
    """Poisson arrivals of (arrival_s, pool index, replicas, hours) for the serving
    workload; landscape sides log-uniform in [128, 2048] over a pool of `pool`."""
    rng = np.random.default_rng(seed)
    sides = [int(round(math.exp(rng.uniform(math.log(128), math.log(2048))))) for _ in range(pool)]
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration_s:
            break
        reqs.append(dict(arrival_s=t, pool_index=int(rng.integers(pool)),
                         n_replicas=int(round(math.exp(rng.uniform(math.log(32), math.log(2048))))),
                         hours=int(rng.integers(12, 73)), seed=int(rng.integers(1 << 62))))
    return sides, reqs


def random_small_case(seed, max_side=24):
    """Small random landscape + weather + parameters for cross-checks on tiny grids."""
    rng = np.random.default_rng(seed)
    rows = int(rng.integers(3, max_side + 1)); cols = int(rng.integers(3, max_side + 1))
    land = heterogeneous_landscape(rows, cols, seed=int(rng.integers(1 << 30)),
                                   nonfuel_frac=float(rng.uniform(0.0, 0.3)))
    hours = int(rng.integers(1, 4))
    weather = weather_stream(hours, seed=int(rng.integers(1 << 30)),
                             ws_mean=float(rng.uniform(0, 45)), ws_sd=10.0)
    params = dict(seed=int(rng.integers(1 << 62)), hours=hours,
                  minutes_per_step=int(rng.choice([1, 2, 3, 5])),
                  ignition_mode=1, ignition_cell=0,
                  ros_sigma=float(rng.choice([0.0, 0.1, 0.5])),
                  ros_threshold=float(rng.choice([0.0, 0.0, 2.0])),
                  burnout_delta=float(rng.choice([0.0, 0.0, 1.5])),
                  const_ros=0.0)
    if rng.random() < 0.3:
        land.unburnable = (rng.random(land.fuel.shape) < 0.1).astype(np.uint8)
    return Workload(land, weather, params)


def digest(*arrays) -> str:
    """sha256 over arrays' dtype, shape and bytes (None counts as absent): a
    checksum of generated inputs, for the manifest in tests/golden."""
    import hashlib
    h = hashlib.sha256()
    for a in arrays:
        if a is None:
            h.update(b"none")
            continue
        a = np.ascontiguousarray(a)
        h.update(str(a.dtype).encode() + str(a.shape).encode())
        h.update(a.tobytes())
    return h.hexdigest()


def workload_digest(w: Workload) -> dict:
    """Checksums of one workload's arrays and its parameters."""
    L = w.landscape
    return {"fuel": digest(L.fuel), "slope": digest(L.slope), "aspect": digest(L.aspect),
            "unburnable": digest(L.unburnable), "weather": digest(w.weather),
            "cell_size": L.cell_size, "params": {k: w.params[k] for k in sorted(w.params)}}
