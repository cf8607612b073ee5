"""CPU oracle for the Cell2Fire fire-growth path (test infrastructure only).

This package is the plain, slow, single-threaded restatement of the method
(Pais et al., arXiv:1905.09317, Algorithm 1 with Secs. 3.1-3.7 and Eqs. 1-4)
that the GPU library is checked against.  Only the test-suite, the smoke
check and the CPU-baseline leg of the benchmark may import it; the product
path never does.  It shares no code with the CUDA library.

The arithmetic lives in ``c2f_oracle.c`` (plain C, binary64, contraction
off); this module compiles it with gcc on first use and wraps it with
ctypes.  ``burn_prob`` (the burn-probability count, Sec. 3.6 / 3.1 outputs)
is a plain numpy sum over replica scars; ``ScenarioOracle`` runs each replica
under its drawn weather scenario (Sec. 3.1 (3)); ``scar_mse`` / ``scar_ssim``
/ ``scar_dnorm`` are the Sec. 4.1 comparison metrics written out on the grids.

Parity status: the FBP surface-spread equations (not printed in the paper)
are "parity unpinned" against their publication; they are pinned only by
closed-form properties.  Everything else is pinned (see tests/).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "c2f_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ROW_LEN = 18
ROW_FIELDS = ("hros", "bros", "lb", "fros", "a", "e", "ux", "uy", "wsv", "wse")


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (no contraction, no fast-math)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
           "-fvisibility=hidden", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64),
        ("hours", C.c_int32),
        ("minutes_per_step", C.c_int32),
        ("ignition_mode", C.c_int32),
        ("ignition_cell", C.c_int32),
        ("ros_sigma", C.c_double),
        ("ros_threshold", C.c_double),
        ("burnout_delta", C.c_double),
        ("ellipse_mode", C.c_int32),
        ("o1_curing_pct", C.c_double),
        ("m1_pc", C.c_double),
        ("const_ros", C.c_double),
        ("burn_hours_min", C.c_int32),
        ("burn_hours_max", C.c_int32),
        ("const_bros", C.c_double),
        ("const_lb", C.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        d, f, i32, u32, u64, i64 = C.c_double, C.c_float, C.c_int32, C.c_uint32, C.c_uint64, C.c_int64
        P = C.POINTER
        lib.or_exp.restype = d; lib.or_exp.argtypes = [d]
        lib.or_log.restype = d; lib.or_log.argtypes = [d]
        lib.or_pow.restype = d; lib.or_pow.argtypes = [d, d]
        lib.or_sincos_deg.restype = None; lib.or_sincos_deg.argtypes = [d, P(d), P(d)]
        lib.or_expf.restype = f; lib.or_expf.argtypes = [f]
        lib.or_logf.restype = f; lib.or_logf.argtypes = [f]
        lib.or_cos_turnsf.restype = f; lib.or_cos_turnsf.argtypes = [f]
        lib.or_philox4x32_10.restype = None
        lib.or_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
        lib.or_noise_factor.restype = f
        lib.or_noise_factor.argtypes = [u64, u32, u32, u32, f]
        lib.or_fbp_cell.restype = None
        lib.or_fbp_cell.argtypes = [C.c_int, d, d, d, d, d, d, d, d, C.c_int, P(d)]
        lib.or_create.restype = C.c_void_p
        lib.or_create.argtypes = [i32, i32, d, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  i32, C.c_void_p, P(Params)]
        lib.or_destroy.restype = None; lib.or_destroy.argtypes = [C.c_void_p]
        lib.or_distances.restype = None; lib.or_distances.argtypes = [C.c_void_p, P(i64)]
        lib.or_cell_row.restype = None; lib.or_cell_row.argtypes = [C.c_void_p, i32, i32, P(d)]
        lib.or_base_inc.restype = None
        lib.or_base_inc.argtypes = [C.c_void_p, i32, i32, P(i64), P(d)]
        lib.or_set_row.restype = None
        lib.or_set_row.argtypes = [C.c_void_p, i32, i32, P(d), d]
        lib.or_ignition_cell.restype = i32; lib.or_ignition_cell.argtypes = [C.c_void_p, i32]
        lib.or_burn_hours.restype = i32; lib.or_burn_hours.argtypes = [C.c_void_p, i32]
        lib.or_scenario_thresholds.restype = C.c_int
        lib.or_scenario_thresholds.argtypes = [i32, P(d), P(u64)]
        lib.or_scenario.restype = i32
        lib.or_scenario.argtypes = [u64, i32, i32, P(u64)]
        for name in ("or_run_replica", "or_run_replica_event"):
            fn = getattr(lib, name)
            fn.restype = C.c_int
            fn.argtypes = [C.c_void_p, i32, C.c_void_p, C.c_void_p, P(i64), P(i32), P(i32)]
        _lib = lib
        return lib


# ---------------------------------------------------------------- math pins
def exp(x: float) -> float: return _load().or_exp(float(x))
def log(x: float) -> float: return _load().or_log(float(x))
def pow(x: float, y: float) -> float: return _load().or_pow(float(x), float(y))  # noqa: A001


def sincos_deg(x: float):
    s, c = C.c_double(), C.c_double()
    _load().or_sincos_deg(float(x), C.byref(s), C.byref(c))
    return s.value, c.value


def expf(x) -> np.float32: return np.float32(_load().or_expf(float(np.float32(x))))
def logf(x) -> np.float32: return np.float32(_load().or_logf(float(np.float32(x))))
def cos_turnsf(u) -> np.float32: return np.float32(_load().or_cos_turnsf(float(np.float32(u))))


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    _load().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def noise_factor(seed: int, replica: int, cell: int, hour: int, sigma: float) -> np.float32:
    return np.float32(_load().or_noise_factor(int(seed), replica, cell, hour,
                                              float(np.float32(sigma))))


def fbp_cell(fuel, slope_pct, aspect_deg, ws, wd_from, ffmc, bui, m1_pc=50.0,
             o1_curing=60.0, ellipse_mode=0) -> dict:
    out = (C.c_double * ROW_LEN)()
    _load().or_fbp_cell(int(fuel), float(slope_pct), float(aspect_deg), float(ws),
                        float(wd_from), float(ffmc), float(bui), float(m1_pc),
                        float(o1_curing), int(ellipse_mode), out)
    row = list(out)
    d = {k: row[i] for i, k in enumerate(ROW_FIELDS)}
    d["ros8"] = np.array(row[10:18])
    return d


# ---------------------------------------------------------------- simulation
def make_params(seed=0, hours=1, minutes_per_step=1, ignition_mode=0, ignition_cell=0,
                ros_sigma=0.0, ros_threshold=0.0, burnout_delta=0.0, ellipse_mode=0,
                o1_curing_pct=60.0, m1_pc=50.0, const_ros=0.0, burn_hours_min=0, burn_hours_max=0,
                const_bros=0.0, const_lb=0.0, **_ignored) -> Params:
    return Params(int(seed), int(hours), int(minutes_per_step), int(ignition_mode),
                  int(ignition_cell), float(ros_sigma), float(ros_threshold),
                  float(burnout_delta), int(ellipse_mode), float(o1_curing_pct),
                  float(m1_pc), float(const_ros), int(burn_hours_min), int(burn_hours_max),
                  float(const_bros), float(const_lb))


class Oracle:
    """One landscape + weather stream + run parameters, simulated replica by replica."""

    def __init__(self, fuel, slope=None, aspect=None, unburnable=None, cell_size=100.0,
                 weather=None, **params):
        self.lib = _load()
        fuel = np.ascontiguousarray(fuel, dtype=np.uint8)
        self.rows, self.cols = fuel.shape
        self.n = self.rows * self.cols
        self._fuel = fuel
        self._slope = None if slope is None else np.ascontiguousarray(slope, dtype=np.float32)
        self._aspect = None if aspect is None else np.ascontiguousarray(aspect, dtype=np.float32)
        self._unb = None if unburnable is None else np.ascontiguousarray(unburnable, dtype=np.uint8)
        w = np.ascontiguousarray(weather, dtype=np.float64).reshape(-1, 4)
        self._weather = w
        self.params = make_params(**params)
        if w.shape[0] < self.params.hours:
            raise ValueError("weather stream shorter than the simulated hours")
        if 60 % self.params.minutes_per_step:
            raise ValueError("minutes_per_step must divide 60")

        def ptr(a):
            return None if a is None else a.ctypes.data_as(C.c_void_p)
        self._h = self.lib.or_create(self.rows, self.cols, float(cell_size), ptr(fuel),
                                     ptr(self._slope), ptr(self._aspect), ptr(self._unb),
                                     int(w.shape[0]), ptr(w), C.byref(self.params))
        self.sph = 60 // self.params.minutes_per_step
        self.steps = self.params.hours * self.sph

    def close(self):
        if getattr(self, "_h", None):
            self.lib.or_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def distances(self):
        d = (C.c_int64 * 8)()
        self.lib.or_distances(self._h, d)
        return list(d)

    def cell_row(self, cell: int, hour: int) -> dict:
        out = (C.c_double * ROW_LEN)()
        self.lib.or_cell_row(self._h, int(cell), int(hour), out)
        row = list(out)
        d = {k: row[i] for i, k in enumerate(ROW_FIELDS)}
        d["ros8"] = np.array(row[10:18])
        return d

    def base_inc(self, cell: int, hour: int):
        b = (C.c_int64 * 8)()
        hr = C.c_double()
        self.lib.or_base_inc(self._h, int(cell), int(hour), b, C.byref(hr))
        return np.array(list(b), dtype=np.int64), hr.value

    def set_row(self, cell: int, hour: int, ros8, hros: float) -> None:
        """Test hook: use the given 8 axis rates (m/min) and HROS as the table row
        of (cell, hour) instead of the oracle's own FBP evaluation."""
        r = (C.c_double * 8)(*[float(v) for v in ros8])
        self.lib.or_set_row(self._h, int(cell), int(hour), r, float(hros))

    def ignition_cell(self, replica: int) -> int:
        return int(self.lib.or_ignition_cell(self._h, int(replica)))

    def burn_hours(self, replica: int) -> int:
        """Burning hours per day of this replica (24: no limit)."""
        return int(self.lib.or_burn_hours(self._h, int(replica)))

    def _run(self, fn, replica):
        scar = np.zeros(self.n, dtype=np.uint8)
        ign = np.zeros(self.n, dtype=np.int32)
        w, ni, ic = C.c_int64(), C.c_int32(), C.c_int32()
        rc = fn(self._h, int(replica), scar.ctypes.data_as(C.c_void_p),
                ign.ctypes.data_as(C.c_void_p), C.byref(w), C.byref(ni), C.byref(ic))
        return {"scar": scar.reshape(self.rows, self.cols),
                "ign": ign.reshape(self.rows, self.cols),
                "work": int(w.value), "n_ignited": int(ni.value), "ignition_cell": int(ic.value)}

    def run_replica(self, replica: int) -> dict:
        """Algorithm 1 stepped period by period (O1)."""
        return self._run(self.lib.or_run_replica, replica)

    def run_replica_event(self, replica: int) -> dict:
        """Label-setting search over ignition steps (O2); equals O1."""
        return self._run(self.lib.or_run_replica_event, replica)


# ---------------------------------------------------------------- weather scenarios
def scenario_thresholds(probs) -> np.ndarray:
    """T_s = floor(2^32 cum_s / total), T_{S-1} = 2^32 (Sec. 3.1, uncertainty (3))."""
    p = np.ascontiguousarray(probs, dtype=np.float64).ravel()
    out = np.zeros(max(p.size, 1), dtype=np.uint64)
    rc = _load().or_scenario_thresholds(int(p.size), p.ctypes.data_as(C.POINTER(C.c_double)),
                                        out.ctypes.data_as(C.POINTER(C.c_uint64)))
    if rc:
        raise ValueError("scenario probabilities must be finite, >= 0 and not all 0")
    return out


def scenario_of(seed: int, replica: int, thresholds) -> int:
    """The scenario replica `replica` runs under: the first s with x0 < T_s."""
    t = np.ascontiguousarray(thresholds, dtype=np.uint64)
    return int(_load().or_scenario(int(seed), int(replica), int(t.size),
                                   t.ctypes.data_as(C.POINTER(C.c_uint64))))


class ScenarioOracle:
    """A request over several weather scenarios (Sec. 3.1, uncertainty (3)):
    replica r runs Algorithm 1 under the weather stream of its drawn scenario
    s(r), with everything else (ignition draw, perturbations, keyed by r)
    as in a single-scenario run."""

    def __init__(self, fuel, slope=None, aspect=None, unburnable=None, cell_size=100.0,
                 weathers=(), probs=(), **params):
        self.thresholds = scenario_thresholds(probs)
        if len(weathers) != self.thresholds.size:
            raise ValueError("one probability per weather scenario")
        self.seed = int(params.get("seed", 0))
        self.oracles = [Oracle(fuel, slope, aspect, unburnable, cell_size=cell_size, weather=w,
                               **params) for w in weathers]

    def scenario(self, replica: int) -> int:
        return scenario_of(self.seed, replica, self.thresholds)

    def ignition_cell(self, replica: int) -> int:
        return self.oracles[0].ignition_cell(replica)

    def base_inc(self, scenario: int, cell: int, hour: int):
        return self.oracles[scenario].base_inc(cell, hour)

    def run_replica(self, replica: int) -> dict:
        s = self.scenario(replica)
        out = self.oracles[s].run_replica(replica)
        out["scenario"] = s
        return out

    def close(self):
        for o in self.oracles:
            o.close()


# ---------------------------------------------------------------- scar comparison
# Sec. 4.1: two simulators' fire scars X^t, Y^t (0-1 matrices, 1 = burned by
# the end of period t) are compared by the mean squared error, the structural
# similarity SSIM of Wang et al. (2004), and, for the final scars, the norm of
# X - Y.  The paper prints SSIM's second denominator factor as
# mu_X^2 + mu_Y^2 + C_2; it is read here as Wang et al.'s sigma_X^2 + sigma_Y^2
# + C_2 (with the printed form SSIM(X, X) would not be 1).  The statistics are
# Wang et al.'s single-window ones over the whole matrix: means, standard
# deviations and covariance with the 1/(N - 1) normalisation, C_1 = (K_1 L)^2,
# C_2 = (K_2 L)^2 with K_1 = 0.01, K_2 = 0.03 and dynamic range L = 1; the norm
# is the Frobenius norm.
SSIM_C1 = (0.01 * 1.0) ** 2
SSIM_C2 = (0.03 * 1.0) ** 2


def scar_at_hour(ign_steps, hour: int, periods_per_hour: int) -> np.ndarray:
    """X^t for t = end of weather hour `hour`: cells ignited at a step <= (hour+1) sph."""
    s = np.asarray(ign_steps)
    return ((s >= 0) & (s <= (hour + 1) * periods_per_hour)).astype(np.float64)


def scar_mse(x, y) -> float:
    """MSE(X, Y) = (1 / nm) sum_ij |X_ij - Y_ij|^2 (Sec. 4.1)."""
    d = np.asarray(x, dtype=np.float64) - np.asarray(y, dtype=np.float64)
    return float(np.mean(np.abs(d) ** 2))


def scar_ssim(x, y) -> float:
    """SSIM(X, Y) = (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2))."""
    x = np.asarray(x, dtype=np.float64).ravel()
    y = np.asarray(y, dtype=np.float64).ravel()
    n = x.size
    mx, my = x.mean(), y.mean()
    vx = np.sum((x - mx) ** 2) / (n - 1)
    vy = np.sum((y - my) ** 2) / (n - 1)
    cxy = np.sum((x - mx) * (y - my)) / (n - 1)
    return float(((2 * mx * my + SSIM_C1) * (2 * cxy + SSIM_C2)) /
                 ((mx * mx + my * my + SSIM_C1) * (vx + vy + SSIM_C2)))


def scar_dnorm(x, y) -> float:
    """delta_norm = ||X - Y|| (Frobenius), for the final scars (Sec. 4.1)."""
    d = np.asarray(x, dtype=np.float64) - np.asarray(y, dtype=np.float64)
    return float(np.linalg.norm(d.ravel()))


def burn_prob(scars) -> np.ndarray:
    """count[c] = number of replicas whose scar contains c (uint32)."""
    s = np.asarray(scars)
    return s.astype(np.uint32).sum(axis=0, dtype=np.uint64).astype(np.uint32)
