"""GB300 (sm_103a) Monte-Carlo fire growth after Cell2Fire (Pais et al., arXiv:1905.09317).

Thin ctypes binding over ``libc2f.so`` (C ABI in ``include/c2f.h``): argument
marshalling only, every step of the fire-growth path runs in the library's
CUDA kernels.  Importing this package does not load the library; the first
call does, and it raises if the library has not been built (``build()``) or
if no CUDA device is present -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .build import LIB as LIB_PATH, build  # noqa: F401

C2F_OK, C2F_EINVAL, C2F_ENOMEM, C2F_ECUDA, C2F_ETIMEOUT = 0, -1, -2, -3, -4
C2F_ENOTFOUND, C2F_EBUSY, C2F_ECANCELED = -5, -6, -7
OUT_SCARS, OUT_IGN_STEPS, OUT_COUNTERS = 1, 2, 8
PROFILE_KERNELS, PROFILE_REPLICAS = 1, 2
TRACE_TABLE, TRACE_REPLICA = 1, 2
_ERR = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ENOTFOUND",
        -6: "EBUSY", -7: "ECANCELED"}


class C2FError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"c2f error {code} ({_ERR.get(code, '?')}): {msg}")
        self.code = code


class WeatherHour(C.Structure):
    _fields_ = [("ws_kmh", C.c_double), ("wd_from_deg", C.c_double),
                ("ffmc", C.c_double), ("bui", C.c_double)]


class SimParams(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64), ("n_replicas", C.c_int32), ("hours", C.c_int32),
        ("minutes_per_step", C.c_int32), ("ignition_mode", C.c_int32),
        ("ignition_cell", C.c_int32), ("ros_sigma", C.c_double),
        ("ros_threshold", C.c_double), ("burnout_delta", C.c_double),
        ("ellipse_mode", C.c_int32), ("o1_curing_pct", C.c_double), ("m1_pc", C.c_double),
        ("const_ros", C.c_double), ("outputs", C.c_uint32),
        ("burn_hours_min", C.c_int32), ("burn_hours_max", C.c_int32),
        ("const_bros", C.c_double), ("const_lb", C.c_double),
    ]


class Tuning(C.Structure):
    """c2f_tuning: the frontier settings the autotuner kept."""
    _fields_ = [("threads", C.c_int32), ("smem_lists", C.c_int32), ("warps_per_sm", C.c_int32),
                ("compact_eighths", C.c_int32), ("list_capacity", C.c_int64), ("frontier_ms", C.c_double),
                ("candidates", C.c_int32)]


class FrontierIO(C.Structure):
    """Device-pointer arguments of c2f_frontier_static (allocation-free frontier step)."""
    _fields_ = [("rows", C.c_int32), ("cols", C.c_int32), ("cell_size_m", C.c_double),
                ("burnable", C.c_void_p), ("base", C.c_void_p), ("hros", C.c_void_p),
                ("ign_cell", C.c_void_p), ("scars", C.c_void_p), ("work", C.c_void_p),
                ("n_ignited", C.c_void_p)]


_lib = None
_lock = threading.Lock()

_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class AllocHooks(C.Structure):
    """c2f_alloc_hooks: device allocations routed through the host framework."""
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", C.c_void_p)]


def torch_alloc_hooks(device: int) -> AllocHooks:
    """Hooks that take the library's device memory from PyTorch's caching
    allocator (stream-ordered on the stream the library names)."""
    import torch

    def alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
        except Exception:
            return None

    def free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    return AllocHooks(_ALLOC_FN(alloc), _FREE_FN(free), None)

# (name, restype, argtypes)
_P = C.POINTER
_SIGS = [
    ("c2f_default_params", None, [_P(SimParams)]),
    ("c2f_create", C.c_int, [_P(C.c_void_p), C.c_int]),
    ("c2f_create_with_hooks", C.c_int, [_P(C.c_void_p), C.c_int, _P(AllocHooks)]),
    ("c2f_set_stream", C.c_int, [C.c_void_p, C.c_void_p]),
    ("c2f_destroy", None, [C.c_void_p]),
    ("c2f_last_error", C.c_char_p, [C.c_void_p]),
    ("c2f_load_landscape", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_double, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, _P(C.c_int32)]),
    ("c2f_set_weather", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]),
    ("c2f_set_weather_scenarios", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                            C.c_void_p]),
    ("c2f_build_ros", C.c_int, [C.c_void_p, C.c_int32, _P(SimParams), C.c_int]),
    ("c2f_get_ros", C.c_int, [C.c_void_p, C.c_int32, _P(SimParams), C.c_int32, C.c_void_p,
                              C.c_void_p, C.c_void_p]),
    ("c2f_get_ros_scenario", C.c_int, [C.c_void_p, C.c_int32, _P(SimParams), C.c_int32, C.c_int32,
                                       C.c_void_p, C.c_void_p, C.c_void_p]),
    ("c2f_simulate", C.c_int, [C.c_void_p, C.c_int32, _P(SimParams), _P(C.c_int32)]),
    ("c2f_simulate_batch", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("c2f_submit", C.c_int, [C.c_void_p, C.c_int32, _P(SimParams), _P(C.c_int32)]),
    ("c2f_pump", C.c_int, [C.c_void_p]),
    ("c2f_poll", C.c_int, [C.c_void_p, C.c_int32, _P(C.c_int32)]),
    ("c2f_wait", C.c_int, [C.c_void_p, C.c_int32]),
    ("c2f_cancel", C.c_int, [C.c_void_p, C.c_int32]),
    ("c2f_set_serving", C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_int64]),
    ("c2f_serving_stats", C.c_int, [C.c_void_p, _P(C.c_int64), _P(C.c_int64), _P(C.c_int32),
                                    _P(C.c_int32)]),
    ("c2f_set_table_mode", C.c_int, [C.c_void_p, C.c_int]),
    ("c2f_burn_prob", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    ("c2f_burn_prob_device", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    ("c2f_burn_prob_scenario", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]),
    ("c2f_get_scars", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    ("c2f_get_replica_scar", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    ("c2f_get_scar_bits", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    ("c2f_get_scars_at_hour", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]),
    ("c2f_get_counters", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("c2f_get_scenarios", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    ("c2f_compare_scars", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("c2f_compare_scars_device", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                           C.c_void_p]),
    ("c2f_set_list_capacity", C.c_int, [C.c_void_p, C.c_int64]),
    ("c2f_set_frontier_config", C.c_int, [C.c_void_p, C.c_int, C.c_int64]),
    ("c2f_set_wait_limit", C.c_int, [C.c_void_p, C.c_int64]),
    ("c2f_test_hold_chunk", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    ("c2f_autotune", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                                _P(C.c_int32), _P(C.c_int32), _P(C.c_double)]),
    ("c2f_autotune_full", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                                     _P(Tuning)]),
    ("c2f_set_compaction", C.c_int, [C.c_void_p, C.c_int32]),
    ("c2f_profile", C.c_int, [C.c_void_p, C.c_int]),
    ("c2f_kernel_times", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("c2f_trace", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    ("c2f_trace_count", C.c_int, [C.c_void_p, _P(C.c_int64)]),
    ("c2f_get_replica_profile", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    ("c2f_fp64_peak", C.c_int, [C.c_void_p, _P(C.c_double)]),
    ("c2f_release", C.c_int, [C.c_void_p, C.c_int32]),
    ("c2f_frontier_static", C.c_int, [C.c_void_p, _P(SimParams), C.c_void_p]),
]
KERNEL_FAMILIES = ("ros_table", "ignite", "frontier", "burn_prob")


def exported_symbols():
    """Names of the C ABI entry points the binding expects the library to export."""
    return [s[0] for s in _SIGS]


def load_library(path: str | None = None):
    """dlopen libc2f.so and declare its signatures (no device call is made)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libc2f.so has not been built ({p}); run "
                               "paper_1905_09317_gb300.build() -- there is no CPU fallback")
        lib = C.CDLL(p)
        for name, res, args in _SIGS:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def default_params(**kw) -> SimParams:
    p = SimParams()
    load_library().c2f_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


class Context:
    """One c2f context on a CUDA device (owns a stream and all device memory)."""

    def __init__(self, device: int = 0, allocator=None):
        """allocator: None (the library's stream-ordered cudaMallocAsync),
        "torch" (device memory from PyTorch's caching allocator) or an
        AllocHooks instance (kept alive by the context)."""
        self.lib = load_library()
        h = C.c_void_p()
        self._hooks = None
        if isinstance(allocator, AllocHooks):
            self._hooks = allocator
            rc = self.lib.c2f_create_with_hooks(C.byref(h), int(device), C.byref(self._hooks))
        elif allocator == "torch":
            self._hooks = torch_alloc_hooks(int(device))
            rc = self.lib.c2f_create_with_hooks(C.byref(h), int(device), C.byref(self._hooks))
        elif allocator is None:
            rc = self.lib.c2f_create(C.byref(h), int(device))
        else:
            raise ValueError(f"unknown allocator {allocator!r}")
        if rc != C2F_OK:
            raise C2FError(rc, f"c2f_create(device={device}) failed (no usable CUDA device?)")
        self.h = h
        self._keep = []

    def _check(self, rc):
        if rc != C2F_OK:
            raise C2FError(rc, self.lib.c2f_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.c2f_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream_ptr: int | None):
        self._check(self.lib.c2f_set_stream(self.h, C.c_void_p(stream_ptr) if stream_ptr else None))

    # ---- inputs
    def load_landscape(self, fuel, slope=None, aspect=None, unburnable=None, cell_size=100.0) -> int:
        fuel = np.ascontiguousarray(fuel, dtype=np.uint8)
        rows, cols = fuel.shape
        s = None if slope is None else np.ascontiguousarray(slope, dtype=np.float32)
        a = None if aspect is None else np.ascontiguousarray(aspect, dtype=np.float32)
        u = None if unburnable is None else np.ascontiguousarray(unburnable, dtype=np.uint8)
        lid = C.c_int32()
        self._check(self.lib.c2f_load_landscape(self.h, rows, cols, float(cell_size), _ptr(fuel),
                                                _ptr(s), _ptr(a), _ptr(u), C.byref(lid)))
        return lid.value

    def set_weather(self, landscape_id: int, weather) -> None:
        w = np.ascontiguousarray(weather, dtype=np.float64).reshape(-1, 4)
        self._check(self.lib.c2f_set_weather(self.h, int(landscape_id), w.shape[0], _ptr(w)))

    def set_weather_scenarios(self, landscape_id: int, weathers, probs) -> None:
        """weathers: (n_scenarios, n_hours, 4); probs: n_scenarios weights."""
        w = np.ascontiguousarray(weathers, dtype=np.float64)
        if w.ndim != 3 or w.shape[2] != 4:
            raise ValueError("weathers must have shape (n_scenarios, n_hours, 4)")
        p = np.ascontiguousarray(probs, dtype=np.float64).ravel()
        if p.size != w.shape[0]:
            raise ValueError("one probability per scenario")
        self._check(self.lib.c2f_set_weather_scenarios(self.h, int(landscape_id), w.shape[0],
                                                       w.shape[1], _ptr(w), _ptr(p)))

    def build_ros(self, landscape_id: int, params: SimParams, force=False) -> None:
        self._check(self.lib.c2f_build_ros(self.h, int(landscape_id), C.byref(params), int(force)))

    def get_ros(self, landscape_id: int, params: SimParams, hour: int, n_cells: int, scenario=0):
        ros8 = np.empty((n_cells, 8), dtype=np.float64)
        hros = np.empty(n_cells, dtype=np.float64)
        base = np.empty((n_cells, 8), dtype=np.int64)
        self._check(self.lib.c2f_get_ros_scenario(self.h, int(landscape_id), C.byref(params),
                                                  int(scenario), int(hour), _ptr(ros8), _ptr(hros),
                                                  _ptr(base)))
        return ros8, hros, base

    # ---- runs
    def simulate(self, landscape_id: int, params: SimParams) -> int:
        sid = C.c_int32()
        self._check(self.lib.c2f_simulate(self.h, int(landscape_id), C.byref(params), C.byref(sid)))
        return sid.value

    def simulate_batch(self, landscape_ids, params_list) -> list[int]:
        n = len(landscape_ids)
        ids = (C.c_int32 * n)(*landscape_ids)
        ps = (SimParams * n)(*params_list)
        out = (C.c_int32 * n)()
        self._check(self.lib.c2f_simulate_batch(self.h, n, ids, ps, out))
        return list(out)

    # ---- serving
    def submit(self, landscape_id: int, params: SimParams) -> int:
        sid = C.c_int32()
        self._check(self.lib.c2f_submit(self.h, int(landscape_id), C.byref(params), C.byref(sid)))
        return sid.value

    def pump(self) -> None:
        self._check(self.lib.c2f_pump(self.h))

    def poll(self, sim_id: int) -> bool:
        d = C.c_int32()
        self._check(self.lib.c2f_poll(self.h, int(sim_id), C.byref(d)))
        return bool(d.value)

    def wait(self, sim_id: int) -> None:
        self._check(self.lib.c2f_wait(self.h, int(sim_id)))

    def cancel(self, sim_id: int) -> None:
        self._check(self.lib.c2f_cancel(self.h, int(sim_id)))

    def set_table_mode(self, eager: bool) -> None:
        """Tables created by simulations: eager (K1 up front) or lazy (filled on demand)."""
        self._check(self.lib.c2f_set_table_mode(self.h, 1 if eager else 0))

    def set_serving(self, max_inflight=3, max_epoch_replicas=1 << 16, hbm_reserve_bytes=2 << 30):
        self._check(self.lib.c2f_set_serving(self.h, int(max_inflight), int(max_epoch_replicas),
                                             int(hbm_reserve_bytes)))

    def serving_stats(self) -> dict:
        e, w, q, r = C.c_int64(), C.c_int64(), C.c_int32(), C.c_int32()
        self._check(self.lib.c2f_serving_stats(self.h, C.byref(e), C.byref(w), C.byref(q), C.byref(r)))
        return dict(epochs=e.value, admission_waits=w.value, queued=q.value, running=r.value)

    # ---- outputs
    def burn_prob(self, sim_id: int, n_cells: int) -> np.ndarray:
        out = np.empty(n_cells, dtype=np.uint32)
        self._check(self.lib.c2f_burn_prob(self.h, int(sim_id), _ptr(out)))
        return out

    def burn_prob_scenario(self, sim_id: int, scenario: int, n_cells: int) -> np.ndarray:
        out = np.empty(n_cells, dtype=np.uint32)
        self._check(self.lib.c2f_burn_prob_scenario(self.h, int(sim_id), int(scenario), _ptr(out)))
        return out

    def burn_prob_device(self, sim_id: int, dev_ptr: int) -> None:
        self._check(self.lib.c2f_burn_prob_device(self.h, int(sim_id), C.c_void_p(dev_ptr)))

    def get_scars(self, sim_id: int, n_replicas: int, n_cells: int, ign_steps=False):
        scars = np.empty((n_replicas, n_cells), dtype=np.uint8)
        ign = np.empty((n_replicas, n_cells), dtype=np.int32) if ign_steps else None
        self._check(self.lib.c2f_get_scars(self.h, int(sim_id), _ptr(scars), _ptr(ign)))
        return scars, ign

    def get_replica_scar(self, sim_id: int, replica: int, n_cells: int, ign_steps=False):
        scar = np.empty(n_cells, dtype=np.uint8)
        ign = np.empty(n_cells, dtype=np.int32) if ign_steps else None
        self._check(self.lib.c2f_get_replica_scar(self.h, int(sim_id), int(replica), _ptr(scar), _ptr(ign)))
        return scar, ign

    def get_scar_bits(self, sim_id: int, n_replicas: int, rows: int, cols: int) -> np.ndarray:
        """(n_replicas, rows, ceil(cols/32)) uint32 words; bit b of word x = column 32x+b."""
        words = np.empty((n_replicas, rows, (cols + 31) // 32), dtype=np.uint32)
        self._check(self.lib.c2f_get_scar_bits(self.h, int(sim_id), _ptr(words)))
        return words

    def get_scars_at_hour(self, sim_id: int, hour: int, n_replicas: int, n_cells: int) -> np.ndarray:
        scars = np.empty((n_replicas, n_cells), dtype=np.uint8)
        self._check(self.lib.c2f_get_scars_at_hour(self.h, int(sim_id), int(hour), _ptr(scars)))
        return scars

    def get_counters(self, sim_id: int, n_replicas: int):
        work = np.empty(n_replicas, dtype=np.int64)
        ign = np.empty(n_replicas, dtype=np.int32)
        cell = np.empty(n_replicas, dtype=np.int32)
        self._check(self.lib.c2f_get_counters(self.h, int(sim_id), _ptr(work), _ptr(ign), _ptr(cell)))
        return work, ign, cell

    def get_scenarios(self, sim_id: int, n_replicas: int) -> np.ndarray:
        out = np.empty(n_replicas, dtype=np.int32)
        self._check(self.lib.c2f_get_scenarios(self.h, int(sim_id), _ptr(out)))
        return out

    def compare_scars(self, sim_x: int, sim_y: int, n_replicas: int, hours: int, hourly=True):
        """Sec. 4.1 metrics: (mse (R, H), ssim (R, H), dnorm (R,)); hourly=False: dnorm only."""
        mse = np.empty((n_replicas, hours), dtype=np.float64) if hourly else None
        ssim = np.empty((n_replicas, hours), dtype=np.float64) if hourly else None
        dn = np.empty(n_replicas, dtype=np.float64)
        self._check(self.lib.c2f_compare_scars(self.h, int(sim_x), int(sim_y), _ptr(mse), _ptr(ssim),
                                               _ptr(dn)))
        return mse, ssim, dn

    def compare_scars_device(self, sim_x: int, sim_y: int, mse_ptr: int, ssim_ptr: int,
                             dnorm_ptr: int) -> None:
        self._check(self.lib.c2f_compare_scars_device(self.h, int(sim_x), int(sim_y),
                                                      C.c_void_p(mse_ptr or None),
                                                      C.c_void_p(ssim_ptr or None),
                                                      C.c_void_p(dnorm_ptr or None)))

    def set_list_capacity(self, cap: int) -> None:
        self._check(self.lib.c2f_set_list_capacity(self.h, int(cap)))

    def set_wait_limit(self, polls: int) -> None:
        """Polls before a frontier wait for a lazy-table chunk gives up (0 = default)."""
        self._check(self.lib.c2f_set_wait_limit(self.h, int(polls)))

    def test_hold_chunk(self, landscape_id: int, hour: int, cell: int, scenario: int = 0) -> None:
        """Test hook: mark the lazy-table chunk of `cell` at `hour` as held by a
        computation that never finishes (exercises the bounded wait)."""
        self._check(self.lib.c2f_test_hold_chunk(self.h, int(landscape_id), int(scenario), int(hour),
                                                 int(cell)))

    def set_frontier_config(self, threads: int, smem_plane_bytes: int) -> None:
        self._check(self.lib.c2f_set_frontier_config(self.h, int(threads), int(smem_plane_bytes)))

    def autotune(self, landscape_ids, params_list, sample_replicas=256):
        """Pick the fastest frontier launch shape for this mix; returns (threads, smem, ms)."""
        n = len(landscape_ids)
        ids = (C.c_int32 * n)(*landscape_ids)
        ps = (SimParams * n)(*params_list)
        t, sm, ms = C.c_int32(), C.c_int32(), C.c_double()
        self._check(self.lib.c2f_autotune(self.h, n, ids, ps, int(sample_replicas), C.byref(t),
                                          C.byref(sm), C.byref(ms)))
        return t.value, sm.value, ms.value

    def autotune_full(self, landscape_ids, params_list, sample_replicas=256) -> dict:
        """All the frontier knobs the autotuner turns, kept on the context; returns them."""
        n = len(landscape_ids)
        ids = (C.c_int32 * n)(*landscape_ids)
        ps = (SimParams * n)(*params_list)
        t = Tuning()
        self._check(self.lib.c2f_autotune_full(self.h, n, ids, ps, int(sample_replicas), C.byref(t)))
        return {f[0]: getattr(t, f[0]) for f in Tuning._fields_}

    def set_compaction(self, eighths: int) -> None:
        self._check(self.lib.c2f_set_compaction(self.h, int(eighths)))

    def profile(self, enable: bool = True, replicas: bool = False) -> None:
        """Kernel-family timing on or off; with `replicas` also the per-replica
        frontier counters (replica_profile)."""
        flags = (PROFILE_KERNELS if enable else 0) | (PROFILE_REPLICAS if replicas else 0)
        self._check(self.lib.c2f_profile(self.h, flags))

    def fp64_peak(self) -> float:
        """Measured FP64 FMA rate of the device, GFLOP/s."""
        g = C.c_double()
        self._check(self.lib.c2f_fp64_peak(self.h, C.byref(g)))
        return g.value

    def trace(self, records_dev_ptr: int | None, capacity: int = 0) -> None:
        """Launch trace into caller device memory (c2f_trace); None turns it off."""
        self._check(self.lib.c2f_trace(self.h, C.c_void_p(records_dev_ptr) if records_dev_ptr else None,
                                       int(capacity)))

    def trace_count(self) -> int:
        n = C.c_int64()
        self._check(self.lib.c2f_trace_count(self.h, C.byref(n)))
        return n.value

    def kernel_times(self) -> dict:
        ms = np.zeros(len(KERNEL_FAMILIES), dtype=np.float64)
        n = np.zeros(len(KERNEL_FAMILIES), dtype=np.int64)
        self._check(self.lib.c2f_kernel_times(self.h, _ptr(ms), _ptr(n)))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_FAMILIES)}

    def replica_profile(self, sim_id: int, n_replicas: int) -> np.ndarray:
        """(n_replicas, 16) frontier counters of a simulation run with profiling on
        (include/c2f.h, c2f_get_replica_profile): total, boundary, send and
        new-cell cycles, visited periods, crossing cells, ignited cells, longest
        burning list, calendar-walk cycles, compactions, crossing rounds,
        new-cell iterations."""
        out = np.empty((n_replicas, 16), dtype=np.int64)
        self._check(self.lib.c2f_get_replica_profile(self.h, int(sim_id), _ptr(out)))
        return out

    def release(self, id_: int) -> None:
        self._check(self.lib.c2f_release(self.h, int(id_)))
