"""Benchmark: Monte-Carlo fire growth on one GB300 (or N, replica-sharded).

Headline (one "step" = one pass of the whole path): the 512x512 heterogeneous
landscape, 24 h hourly weather, 1000 replicas with random ignitions and
lognormal(0, 0.1) ROS noise -- ROS table (K1), ignition (K2), frontier (K3)
and burn-probability counts (K4).  Metric: cell-updates/s, the number of
(burning cell, fire period) pairs of Algorithm 1 per second, summed over
replicas; replicas/s is reported beside it.  Steps are pipelined (the next
steps' tables overlap the current frontier).

The same JSON line also carries, each with its own timing and clock record:
  plain    the same step as one synchronous c2f_simulate at a time (one
           request per launch); its per-kernel times feed the roofline entries;
  batched  64 landscapes of 64^2..2048^2 cells, 16..4096 replicas, 48 h: one
           call per landscape vs one batched call (tables and frontiers in one
           CUDA graph);
  served   Poisson arrivals (50/s; a 10 s window, --serve-window) over a pool
           of 16 landscapes, served with submit/poll (continuous batching):
           throughput and p50/p99 latency, and a capacity comparison with the
           first requests all waiting (served vs one synchronous call each);
  large    4096^2 cells, 72 h with a 90-degree wind shift, 256 replicas.
Their inputs are generated in spawned host processes once the headline
workload's timings are done, and all of them before the first section is
timed: the thread that issues GPU work must not wait for a host core.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own 1000 replicas (replica ids offset by
rank), so per-GPU work is fixed (weak scaling) and no collective touches the
data path; the timing is max-over-ranks.  --gpus must equal the number of
processes launched (it is refused otherwise).

Other workloads (one GPU; each prints its own JSON line):
  --workload batch | serve | large   the sections above on their own (serve
                     with 60 s of arrivals, --duration)
  --workload scenarios  the 512^2 landscape under 8 weather scenarios x 24 h with
                     probabilities; each of 1000 replicas draws its scenario.
  --workload compare the Sec. 4.1 scar comparison (hourly MSE / SSIM, final
                     norm) of two 1000-replica runs of the 512^2 workload.
  --workload burnhours  the 512^2 landscape over 48 h with fires that burn only
                     6-12 hours a day (drawn per replica), beside the same
                     replicas with no limit.
  --workload replica-profile  the headline workload's frontier once with the
                     per-replica counters on: cycles per visited period by phase.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import c2f_synth as S  # noqa: E402

WORKLOAD = "512x512 heterogeneous FBP landscape, 100 m cells, 24 h hourly weather, " \
           "1000 replicas, random ignitions, lognormal(0,0.1) ROS noise, 1-min clock"
METRIC = "cell-updates/s"


# ------------------------------------------------------------------ helpers
_ORACLES = {}


def _oracle_chunk(args):
    """(spawned process) run oracle replicas; returns (sum of work, replicas)."""
    side, hours, replicas = args
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import c2f_synth as S2
    import oracle
    key = (side, hours)
    if key not in _ORACLES:
        w = S2.config2(side=side, hours=hours)
        L = w.landscape
        _ORACLES[key] = oracle.Oracle(L.fuel, L.slope, L.aspect, cell_size=L.cell_size,
                                      weather=w.weather, **w.params)
    o = _ORACLES[key]
    tot = 0
    for r in replicas:
        tot += o.run_replica(r)["work"]
    return tot, len(replicas)


def _workload_of(key):
    """Workloads by name, rebuilt from their seeds inside a worker process."""
    import c2f_synth as S2
    if key[0] == "large":
        return S2.config4()
    if key[0] == "batch":
        return S2.config3_workload(S2.config3_specs()[key[1]])
    raise KeyError(key)


def _oracle_sample_chunk(items):
    """(spawned process) oracle replicas of named workloads: [(key, replica), ...]."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    tot, t_run = 0, 0.0
    cur, o = None, None
    for key, r in sorted(items):
        if key != cur:   # one oracle at a time: large landscapes reserve much memory
            if o is not None:
                o.close()
            w = _workload_of(key)
            L = w.landscape
            o = oracle.Oracle(L.fuel, L.slope, L.aspect, cell_size=L.cell_size, weather=w.weather,
                              **w.params)
            cur = key
        t0 = time.perf_counter()
        tot += o.run_replica(r)["work"]
        t_run += time.perf_counter() - t0
    if o is not None:
        o.close()
    return tot, t_run


def cpu_oracle_sample_rate(items, procs: int):
    """Oracle cell-updates/s on a sample of (workload, replica) items, one process per
    core; inputs are built outside the timing, the rate is the sampled work over the
    slowest process's replica time."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    chunks = [items[p::procs] for p in range(procs)]
    chunks = [c for c in chunks if c]
    with mp.get_context("spawn").Pool(len(chunks)) as pool:
        res = pool.map(_oracle_sample_chunk, chunks)
    work = sum(r[0] for r in res)
    t = max(r[1] for r in res)
    return work / t, work, t, len(chunks)


def cpu_oracle_rate(n_replicas_sample: int, procs: int):
    """Oracle (single-threaded C, one process per core) on a replica sample."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    chunks = [list(range(p, n_replicas_sample, procs)) for p in range(procs)]
    chunks = [c for c in chunks if c]
    with ctx.Pool(len(chunks)) as pool:
        pool.map(_oracle_chunk, [(512, 24, [])] * len(chunks))   # build inputs outside the timing
        t0 = time.perf_counter()
        res = pool.map(_oracle_chunk, [(512, 24, c) for c in chunks])
        dt = time.perf_counter() - t0
    work = sum(r[0] for r in res)
    return work / dt, work, dt, len(chunks)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.skip = 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)            # sampling is running before the timed region starts
            self.skip = len(self.lines)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.skip:] or self.lines[-1:]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ multi-rank pieces
def rank_seed(seed: int, rank: int) -> int:
    """Each rank runs its own replicas: the run seed is offset per rank (the
    replica index keys the counter, the seed keys Philox), so no replica of one
    rank repeats another rank's."""
    return int(seed) + 7919 * int(rank)


def max_over_ranks(x: float, world: int, device) -> float:
    """The slowest rank's time (all_reduce MAX; identity for one rank)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: int, world: int, steps: int, seconds: float) -> float:
    """Units all ranks processed over the slowest rank's time (weak scaling)."""
    return units_per_rank_step * world * steps / seconds


def gpus_mismatch(gpus: int, world: int):
    """--gpus N must be what the launcher started: one process per GPU under
    torchrun (WORLD_SIZE = N), or a single process for N = 1.  A mismatch would
    time a different number of GPUs than the line claims, so it is refused."""
    if gpus < 1:
        return f"--gpus must be >= 1 (got {gpus})"
    if gpus != world:
        return (f"--gpus {gpus} but {world} process(es) were launched (WORLD_SIZE={world}); run "
                f"N > 1 as: python -m torch.distributed.run --nproc-per-node {gpus} bench.py --gpus {gpus} ...")
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


# ------------------------------------------------------------------ workload generation
def _gen_batch(i):
    """(spawned process) landscape i of the 64-landscape batch."""
    return S.config3_workload(S.config3_specs()[i])


def _gen_large():
    """(spawned process) the 4096^2 workload."""
    return S.config4()


def _gen_serve_land(side, seed):
    """(spawned process) one landscape of the request stream's pool."""
    return S.heterogeneous_landscape(side, seed=seed)


def _low_priority():
    """(spawned process initializer) the lowest CPU priority, so that the thread
    that issues GPU work keeps its core when the host is busy."""
    try:
        os.nice(19)
    except OSError:
        pass


class WorkloadPool:
    """The batch, request-stream and 4096^2 inputs, generated in spawned
    processes (host numpy only, one thread each, lowest priority, two cores
    left free)."""

    def __init__(self, serve_rate, serve_window):
        import concurrent.futures as cf
        import multiprocessing as mp
        workers = max(1, min(16, (os.cpu_count() or 1) - 2))
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(v, "1")   # one thread per generating process
        self.ex = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"),
                                         initializer=_low_priority)
        self.f_large = self.ex.submit(_gen_large)
        self.specs = S.config3_specs()
        self.f_batch = [self.ex.submit(_gen_batch, i) for i in range(len(self.specs))]
        self.sides, self.reqs = S.serving_requests(rate=serve_rate, duration_s=serve_window)
        self.f_serve = [self.ex.submit(_gen_serve_land, side, 500 + i) for i, side in enumerate(self.sides)]

    def batch(self):
        return [f.result() for f in self.f_batch]

    def large(self):
        return self.f_large.result()

    def serve(self):
        return self.sides, self.reqs, [f.result() for f in self.f_serve]

    def close(self):
        self.ex.shutdown(wait=True, cancel_futures=True)


def _section(fn, *a):
    """One extra section of the default line; a failure is reported, not hidden."""
    try:
        return fn(*a)
    except Exception as e:   # the headline line is still printed, with the error beside it
        return {"error": f"{type(e).__name__}: {e}"}


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    extras_on = world == 1 and not args.no_extras
    pool = None
    import torch
    import paper_1905_09317_gb300 as c2f

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c2f.build()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    w = S.config2(n_replicas=args.replicas)
    L = w.landscape
    n = L.fuel.size
    R = w.params["n_replicas"]
    keys = {f[0] for f in c2f.SimParams._fields_}
    params = c2f.default_params(**{k: v for k, v in w.params.items() if k in keys})
    params.seed = rank_seed(params.seed, rank)       # each rank: its own replicas

    ctx = c2f.Context(local_rank)
    if args.frontier_threads:
        ctx.set_frontier_config(args.frontier_threads, args.smem_plane_bytes)
    pipe_warps = None
    if not args.frontier_threads and not args.serial:
        # pipelined steps: size each warp's shared memory for one warp per SM
        # more than a step's own replicas need, so that the next step's
        # frontier starts beside the current one's last replicas
        pipe_warps = -(-R // sms) + 1
        ctx.set_frontier_config(32, pipe_warps)
    # the context issues its work (K1, K4, uploads) on this stream and the
    # timing events are recorded on it; frontier epochs run on the context's own
    # epoch streams and are waited for on the host before a step's K4
    stream = torch.cuda.Stream(dev)
    ctx.set_stream(stream.cuda_stream)
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
    ctx.set_weather(lid, w.weather)
    counts_dev = torch.empty(n, dtype=torch.int32, device=dev)

    table_mode = 2 if args.lazy_tables else 1
    ctx.set_table_mode(not args.lazy_tables)

    def step():
        ctx.build_ros(lid, params, force=table_mode)            # a1 + a2 (K1; on demand when lazy)
        sid = ctx.simulate(lid, params)                         # a3..a8 (K2, K3)
        ctx.burn_prob_device(sid, counts_dev.data_ptr())        # a9 (K4)
        return sid

    # Pipelined steps: each step's table is built (K1, context stream) while the
    # previous step's frontier runs (its own stream, submitted asynchronously);
    # the work of a step is the same as in the serial form.
    depth = max(2, args.depth)                  # steps in flight
    ctx.set_serving(max_inflight=depth, max_epoch_replicas=R, hbm_reserve_bytes=0)

    def run_steps(k):
        if args.serial:
            done = []
            for _ in range(k):
                sid = step()
                if done:
                    ctx.release(done.pop())   # as in the pipelined form: the last step is kept
                done.append(sid)
            return done
        done, inflight = [], []

        def retire():
            sid = inflight.pop(0)
            ctx.wait(sid)
            ctx.burn_prob_device(sid, counts_dev.data_ptr())    # a9 (K4)
            # a step's result is its counts: the simulation (and the table only it
            # still holds) is released at once, as a serving caller would, so the
            # next builds reuse that memory (freed after K4 has read the scars);
            # the last step is kept for its work counters
            if done:
                ctx.release(done.pop())
            done.append(sid)

        for _ in range(k):
            ctx.build_ros(lid, params, force=table_mode)        # a1 + a2 (K1)
            inflight.append(ctx.submit(lid, params))            # a3..a8 (K2, K3), asynchronous
            if len(inflight) >= depth:
                retire()
        while inflight:
            retire()
        return done

    # warm-up (also fixes the deterministic work count of the step)
    for sid in run_steps(max(args.warmup, 1)):
        work, _, _ = ctx.get_counters(sid, R)
        ctx.release(sid)
    work_per_step = int(work.sum())

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    ctx.profile(True)
    ctx.kernel_times()
    sampler = ClockSampler(local_rank)
    barrier()
    with sampler:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        sids = run_steps(args.steps)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    kt = ctx.kernel_times()
    ctx.profile(False)
    last_work, _, _ = ctx.get_counters(sids[-1], R)
    assert int(last_work.sum()) == work_per_step, "work count changed between steps"
    for s in sids:
        ctx.release(s)
    ms_max = max_over_ranks(ms, world, dev)

    # e2e: host buffers through the C ABI, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        host_counts = np.empty(n, dtype=np.uint32)
        h2d = L.fuel.nbytes + L.slope.nbytes + L.aspect.nbytes + w.weather.nbytes
        e2e_steps = max(1, args.steps)   # as many steps as the device-resident timing
        # every step: the landscape and weather uploaded from host arrays, the
        # simulation submitted, the burn counts read back to the host; steps
        # pipelined like the device-resident ones (unless --serial)
        barrier()
        t0 = time.perf_counter()
        pending = []

        def retire_e2e():
            s2, l2 = pending.pop(0)
            ctx.wait(s2)
            host_counts[:] = ctx.burn_prob(s2, n)
            ctx.release(s2)
            ctx.release(l2)

        for _ in range(e2e_steps):
            l2 = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
            ctx.set_weather(l2, w.weather)
            if args.serial:
                s2 = ctx.simulate(l2, params)
                host_counts[:] = ctx.burn_prob(s2, n)
                ctx.release(s2)
                ctx.release(l2)
                continue
            pending.append((ctx.submit(l2, params), l2))
            if len(pending) >= depth:
                retire_e2e()
        while pending:
            retire_e2e()
        torch.cuda.synchronize(dev)
        e2e_s = time.perf_counter() - t0
        e2e_max = max_over_ranks(e2e_s, world, dev)
        e2e = dict(value=whole_job_rate(work_per_step, world, e2e_steps, e2e_max), unit=METRIC,
                   h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(host_counts.nbytes),
                   steps=e2e_steps)

    # plain: the same step as one synchronous c2f_simulate at a time (one
    # request per launch, nothing overlapped), timed with CUDA events; then a
    # few such steps with per-kernel events: each kernel's duration when it runs
    # by itself (the roofline's timing)
    if pipe_warps:
        ctx.set_frontier_config(32, 1)   # the default sizing for a launch that runs alone
    plain_steps = max(3, args.plain_steps)
    sampler_plain = ClockSampler(local_rank)
    barrier()
    with sampler_plain:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(plain_steps):
            ctx.release(step())
        ev1.record(stream)
        barrier()
    ms_plain = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    ctx.profile(True)
    ctx.kernel_times()
    for _ in range(3):
        ctx.release(step())
    kt_alone = ctx.kernel_times()
    ctx.profile(False)
    fp64_peak = ctx.fp64_peak()   # outside the timed regions: the table kernel's FP64 roofline
    trace = None
    if world == 1 and not args.serial and not args.lazy_tables and args.trace_steps > 0:
        # outside the timed regions: how K1 and K3 share the device, one step alone
        # and then pipelined steps (launch trace, c2f_trace)
        trace = _section(pipeline_trace, ctx, torch, dev, step, run_steps, sms, args.trace_steps,
                         args.trace_out)
    ctx.release(lid)
    ctx.close()

    # the extra sections' inputs: generated on the host cores only now, after every
    # timing of the headline workload (the thread that issues its steps must not
    # wait for a core), and all of them before the first section is timed
    sections_in = None
    if extras_on and rank == 0:
        pool = WorkloadPool(args.rate, args.serve_window)
        sections_in = (pool.batch(), pool.serve(), pool.large())
        pool.close()

    out = None
    if rank == 0:
        value = whole_job_rate(work_per_step, world, args.steps, ms_max / 1e3)
        peaks = measured_peaks()
        clocks = sampler.summary()
        plain = {"value": whole_job_rate(work_per_step, world, plain_steps, ms_plain / 1e3), "unit": METRIC,
                 "ms_per_step": ms_plain / plain_steps, "steps": plain_steps,
                 "replicas_per_s": R * world * plain_steps / (ms_plain / 1e3),
                 "schedule": "one synchronous c2f_simulate per step (one request per launch), the table "
                             "rebuilt every step, nothing overlapped",
                 "kernel_ms_alone": {k: v[0] / max(v[1], 1) * (2 if k == "ros_table" else 1)
                                     for k, v in kt_alone.items()},
                 "clocks": sampler_plain.summary()}
        roof = frontier_roofline(kt_alone, w, work_per_step, peaks, sms,
                                 plain["clocks"].get("sm_mhz") or clocks.get("sm_mhz"))
        roof_k1 = roofline_table(kt_alone, w, fp64_peak)
        launches = int(sum(v[1] for v in kt.values()))   # every kernel of the timed steps
        extras = {}
        if extras_on:
            batch_in, serve_in, large_in = sections_in
            extras["batched"] = _section(batch_measure, args, batch_in, pool.specs, 2, 1, local_rank)
            extras["served"] = _section(serve_measure, args, *serve_in, local_rank)
            extras["large"] = _section(large_measure, args, large_in, 2, local_rank)
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            procs = os.cpu_count() or 1
            rate, cw, cdt, used = cpu_oracle_rate(args.cpu_sample, procs)
            cpu = dict(value=rate, unit=METRIC, cores=used, kind="oracle",
                       sample=f"replicas 0..{args.cpu_sample - 1} of the workload, "
                              f"{used} single-threaded oracle processes, {cdt:.1f} s wall")
        out = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "replicas_per_gpu": R, "hours": 24,
                       "cells": int(n), "cell_updates_per_step_per_gpu": work_per_step,
                       "l2": "inputs larger than L2 (ROS table 453 MB rebuilt every step)",
                       "parallelism": f"replica-sharded x{world}",
                       "schedule": "serial" if args.serial else
                       f"pipelined, {max(2, args.depth)} steps in flight: the next steps' tables (K1) "
                       "overlap the current frontier (K3)",
                       "tables": "on demand in K3" if args.lazy_tables else "K1, every row",
                       "frontier_smem": (f"sized for {pipe_warps} warps per SM (one more than a step's "
                                         "replicas need: the next step's frontier starts beside it)")
                       if pipe_warps else "library default"},
            "replicas_per_s": R * world * args.steps / (ms_max / 1e3),
            "kernel_event_ms_per_step": {k: v[0] / args.steps for k, v in kt.items()},
            "kernel_event_note": "sums of each family's event brackets in the pipelined steps; the "
                                 "brackets of overlapping steps overlap, so these are not durations "
                                 "(plain.kernel_ms_alone are)",
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "roofline_table_kernel": roof_k1,
            "clocks": clocks,
            "plain": plain,
            "pipeline_trace": trace,
            **extras,
        }
        if extras_on and "error" not in extras.get("batched", {}) and "error" not in extras.get("served", {}):
            out["batched_over_plain"] = extras["batched"]["batched_over_plain"]
            out["served_over_plain"] = extras["served"]["capacity"]["served_over_plain"]
    return out


def timeline(rec, sms):
    """Per-build and per-simulation spans of a launch trace (c2f_trace records:
    kind | SM << 8 | aux << 32, tag, start ns, end ns), the K1 builds' resident
    CTAs per SM, the replicas resident beside them, and replica durations."""
    import numpy as np
    kind = (rec[:, 0] & 0xFF).astype(np.int64)
    tag = rec[:, 1].astype(np.int64)
    t0 = rec[:, 2].astype(np.float64)
    t1 = rec[:, 3].astype(np.float64)
    base = t0.min()
    t0 = (t0 - base) / 1e6                      # ms
    t1 = (t1 - base) / 1e6
    tab, rep = kind == 1, kind == 2
    builds = []
    for tg in np.unique(tag[tab]):
        m = tab & (tag == tg)
        builds.append((t0[m].min(), t1[m].max(), float((t1[m] - t0[m]).sum())))
    builds.sort()
    sims = []
    for tg in np.unique(tag[rep]):
        m = rep & (tag == tg)
        d = t1[m] - t0[m]
        sims.append((t0[m].min(), t1[m].max(), float(np.median(d)), float(d.max())))
    sims.sort()
    out = {"builds": len(builds), "simulations": len(sims)}
    if builds:
        spans = [b[1] - b[0] for b in builds]
        busy = sum(b[2] for b in builds)
        out["k1_ms"] = float(np.median(spans))
        out["k1_ctas_per_sm"] = busy / sum(spans) / sms
        if len(builds) > 1:
            out["k1_gap_ms"] = float(np.median([builds[i + 1][0] - builds[i][1] for i in range(len(builds) - 1)]))
            out["build_period_ms"] = (builds[-1][0] - builds[0][0]) / (len(builds) - 1)
        # replica-time inside the build windows, per SM
        inside = 0.0
        rs, re_ = t0[rep], t1[rep]
        for b0, b1, _ in builds:
            inside += float(np.clip(np.minimum(re_, b1) - np.maximum(rs, b0), 0, None).sum())
        out["replicas_per_sm_during_k1"] = inside / sum(spans) / sms
    if sims:
        out["replica_ms_median"] = float(np.median([x[2] for x in sims]))
        out["replica_ms_max"] = float(max(x[3] for x in sims))
        out["frontier_span_ms"] = float(np.median([x[1] - x[0] for x in sims]))
    lines = []
    for b in builds:
        lines.append((b[0], f"K1 build   {b[0]:9.3f} .. {b[1]:9.3f} ms  span {b[1] - b[0]:6.3f} ms  "
                            f"{b[2] / (b[1] - b[0]) / sms:5.2f} CTAs/SM"))
    for x in sims:
        lines.append((x[0], f"frontier   {x[0]:9.3f} .. {x[1]:9.3f} ms  span {x[1] - x[0]:6.3f} ms  "
                            f"replica median {x[2]:6.3f} max {x[3]:6.3f} ms"))
    return out, [t for _, t in sorted(lines, key=lambda x: x[0])]


def pipeline_trace(ctx, torch, dev, step, run_steps, sms, k, out_path):
    """One step alone, then k pipelined steps, under the launch trace."""
    import numpy as np
    cap = 1 << 21
    buf = torch.empty(cap * 4, dtype=torch.int64, device=dev)

    def traced(fn):
        torch.cuda.synchronize(dev)
        ctx.trace(buf.data_ptr(), cap)
        sids = fn()
        torch.cuda.synchronize(dev)
        cnt = ctx.trace_count()
        ctx.trace(None)
        for s in sids:
            ctx.release(s)
        return buf.view(-1, 4)[:min(cnt, cap)].cpu().numpy().view(np.uint64), cnt

    rec_a, na = traced(lambda: [step()])
    rec_p, npp = traced(lambda: run_steps(k))
    alone, lines_a = timeline(rec_a, sms)
    piped, lines_p = timeline(rec_p, sms)
    if out_path:
        with open(out_path, "w") as f:
            f.write(f"# launch trace: one step alone ({na} records)\n")
            f.write("\n".join(lines_a) + "\n")
            f.write(f"# {k} pipelined steps ({npp} records)\n")
            f.write("\n".join(lines_p) + "\n")
            f.write(json.dumps({"alone": alone, "pipelined": piped}) + "\n")
    return {"steps": k, "alone": alone, "pipelined": piped,
            "note": "c2f_trace records (globaltimer), outside the timed regions: K1 build spans and "
                    "gaps, resident K1 CTAs and replicas per SM while builds run, replica durations"}


def frontier_roofline(kt_alone, w, work_per_step, peaks, sms, sm_mhz):
    """K3 against what bounds it, from its duration when a step runs by itself.

    The event-driven frontier moves about 2 B of DRAM per cell-update (ncu), so
    HBM is far from its limit; it is bound by the latency of one warp per
    replica.  achieved / frac: DRAM bytes per launch (ncu, scaled by the
    replicas) over the launch's duration, against the measured copy bandwidth.
    issue: warp instructions per launch (ncu, per cell-update) over the
    duration, against every scheduler issuing every cycle.  The period-by-
    period method's 194 B per cell-update is kept as period_method_equiv_gbs:
    the bandwidth that method would need for this throughput."""
    ms, launches = kt_alone["frontier"]
    if launches == 0:
        return None
    per_launch_s = ms / launches / 1e3
    hbm = peaks.get("hbm_gbs", 6800.0)
    R = w.params["n_replicas"]
    traffic = FRONTIER_DRAM_BYTES_PER_REPLICA * R
    ach = traffic / per_launch_s / 1e9
    mhz = float(sm_mhz or peaks.get("sm_max_mhz", 2070.0))
    inst = FRONTIER_WARP_INST_PER_UPDATE * work_per_step
    issue_peak = sms * 4 * mhz * 1e6          # warp instructions per second, 4 schedulers per SM
    return {"kernel": "k_frontier_w1", "bound": "latency", "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm, "traffic": traffic, "ms_per_launch": per_launch_s * 1e3,
            "timing": "K3 launches of plain steps (one step at a time), CUDA events",
            "traffic_source": FRONTIER_PROFILE_NOTE,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
            "issue": {"warp_inst_per_launch": inst, "achieved_ginst_per_s": inst / per_launch_s / 1e9,
                      "peak_ginst_per_s": issue_peak / 1e9, "frac": inst / per_launch_s / issue_peak,
                      "peak_source": f"{sms} SMs x 4 schedulers x {mhz:.0f} MHz (SM clock sampled under load)"},
            "l2": {"bytes_per_launch": FRONTIER_L2_BYTES_PER_REPLICA * R,
                   "achieved_gbs": FRONTIER_L2_BYTES_PER_REPLICA * R / per_launch_s / 1e9,
                   "pct_of_peak_in_capture": FRONTIER_L2_PCT_IN_CAPTURE,
                   "source": "ncu lts__t_sectors of the same 200-replica launch, scaled by replicas"},
            "period_method_equiv_gbs": FRONTIER_BYTES_PER_UPDATE * work_per_step / per_launch_s / 1e9,
            "period_method_note": "194 B per cell-update (8 x 8 B progress read and written, 8 x 8 B rates, "
                                  "neighbour bits) is what the period-by-period method would move; the "
                                  "event-driven kernel does not move it"}


def roofline_table(kt, w, fp64_peak):
    """K1 against the device's FP64 rate (binary64 flops per cell-hour, ncu)."""
    ms, launches = kt["ros_table"]
    if launches == 0:
        return None
    n = w.landscape.fuel.size
    H = w.params["hours"]
    flops = FP64_OPS_PER_CELL_HOUR * n * H
    peak = fp64_peak or FP64_PEAK_GFLOPS
    # the family brackets two launches per table build (hour prep, then the table kernel)
    ach = flops / (ms / max(launches // 2, 1) / 1e3) / 1e9
    return {"kernel": "k_ros_table", "bound": "alu", "achieved": ach, "peak": peak,
            "unit": "GFLOP/s (fp64)", "frac": ach / peak, "traffic": None,
            "peak_source": "measured: c2f_fp64_peak (FP64 FMA chains, this run)" if fp64_peak else
                           "derived: 152 SMs x 2 DFMA/clk x 2 flop x SM clock"}


# Algorithmic and measured figures.  Frontier: bytes per cell-update of the
# period-by-period method (8 x 8 B progress read and written, 8 x 8 B rates
# read, ~2 B of neighbour state); DRAM bytes per replica and warp instructions
# per cell-update from ncu on the 512^2 x 24 h workload.  ROS table: binary64
# flops per cell-hour (2 x DFMA + DMUL + DADD from ncu's instruction counts over
# cells x hours).  FP64 peak: 152 SMs x 2 DFMA per clock x 2 flop x 2.07 GHz.
FRONTIER_BYTES_PER_UPDATE = 194.0
FRONTIER_DRAM_BYTES_PER_REPLICA = (96.998e6 + 14.878e6) / 200   # 200-replica launch: read + write
FRONTIER_WARP_INST_PER_UPDATE = 214.105e6 / 43484764             # warp instructions / cell-updates
FRONTIER_L2_BYTES_PER_REPLICA = 20432252 * 32 / 200                 # lts__t_sectors x 32 B / replicas
FRONTIER_L2_PCT_IN_CAPTURE = 0.43                                   # lts__t_sectors % of peak, same capture
FRONTIER_PROFILE_NOTE = "ncu dram__bytes_read+write and smsp__inst_executed of a 200-replica launch, " \
                        "scaled by replicas / cell-updates"
FP64_OPS_PER_CELL_HOUR = 364.0      # ncu: (2 x DFMA + DMUL + DADD) / (cells x hours)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07   # SMs x DFMA/clk x flop/DFMA x GHz


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    """The CPU oracle on the host cores, on a bounded replica sample per step."""
    if rank != 0:
        return None
    procs = os.cpu_count() or 1
    rates, works, dts = [], [], []
    for _ in range(max(args.warmup, 0)):
        cpu_oracle_rate(min(args.ref_sample, procs), procs)
    for _ in range(args.steps):
        rate, cw, cdt, used = cpu_oracle_rate(args.ref_sample, procs)
        rates.append(rate); works.append(cw); dts.append(cdt)
    value = sum(works) / sum(dts)
    sample = (f"replicas 0..{args.ref_sample - 1} of the workload per step, "
              f"{used} single-threaded oracle processes")
    return {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(dts) / len(dts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": used, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------ other workloads
def _params_of(c2f, w, **over):
    keys = {f[0] for f in c2f.SimParams._fields_}
    d = {k: v for k, v in w.params.items() if k in keys}
    d.update(over)
    return c2f.default_params(**d)


def batch_measure(args, ws, specs, steps, warmup, device=0):
    """64-landscape batch: plain (one c2f_simulate per landscape) vs batched (one
    c2f_simulate_batch), tables rebuilt every pass, the same autotuned launch shape."""
    import torch
    import paper_1905_09317_gb300 as c2f
    c2f.build()
    ctx = c2f.Context(device)
    ctx.set_table_mode(not args.lazy_tables)
    if args.frontier_threads:
        ctx.set_frontier_config(args.frontier_threads, args.smem_plane_bytes)
    lids = []
    for w in ws:
        L = w.landscape
        lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
        ctx.set_weather(lid, w.weather)
        lids.append(lid)
    ps = [_params_of(c2f, w) for w in ws]
    ns = [w.landscape.fuel.size for w in ws]
    tuned = None
    if not args.frontier_threads:   # frontier settings chosen by the autotuner on a scaled-down copy
        t0 = time.perf_counter()
        tuned = ctx.autotune_full(lids, ps, sample_replicas=args.tune_sample)
        tuned["tuning_s"] = time.perf_counter() - t0
        tuned["sample_replicas"] = args.tune_sample

    def plain():
        sids = []
        for lid, p, w in zip(lids, ps, ws):
            ctx.set_weather(lid, w.weather)          # the table is rebuilt inside the step
            sids.append(ctx.simulate(lid, p))
        return sids

    def batched():
        for lid, w in zip(lids, ws):
            ctx.set_weather(lid, w.weather)
        return ctx.simulate_batch(lids, ps)

    # the same two paths with every table kept from the previous pass (built once,
    # as a served landscape's table is): what batching does for the frontiers
    def plain_resident():
        return [ctx.simulate(lid, p) for lid, p in zip(lids, ps)]

    def batched_resident():
        return ctx.simulate_batch(lids, ps)

    out = {}
    work = None
    for name, fn in (("plain", plain), ("batched", batched), ("plain_resident", plain_resident),
                     ("batched_resident", batched_resident)):
        for _ in range(max(warmup, 1)):
            for sid in fn():
                ctx.release(sid)
        torch.cuda.synchronize()
        sampler = ClockSampler(device)
        with sampler:
            t0 = time.perf_counter()
            for _ in range(steps):
                sids = fn()
                for sid, n in zip(sids, ns):
                    ctx.burn_prob(sid, n)
                wk = sum(int(ctx.get_counters(sid, p.n_replicas)[0].sum()) for sid, p in zip(sids, ps))
                for sid in sids:
                    ctx.release(sid)
                assert work is None or wk == work, "work count differs between plain and batched"
                work = wk
            dt = (time.perf_counter() - t0) / steps
        # one more pass, outside the timing, with per-kernel device times
        ctx.profile(True)
        ctx.kernel_times()
        for sid in fn():
            ctx.release(sid)
        kt = ctx.kernel_times()
        ctx.profile(False)
        out[name] = dict(s_per_step=dt, cell_updates_per_s=work / dt,
                         replicas_per_s=sum(p.n_replicas for p in ps) / dt,
                         kernel_ms={k: v[0] for k, v in kt.items()},
                         kernel_launches={k: v[1] for k, v in kt.items()},
                         clocks=sampler.summary())
    ctx.close()
    return {"value": out["batched"]["cell_updates_per_s"], "unit": METRIC, "steps": steps, "warmup": warmup,
            "config": {"workload": "batch of 64 landscapes, sides log-uniform 64..2048 cells, replicas "
                                   "log-uniform 16..4096, 48 h weather, random ignitions, lognormal(0,0.1) "
                                   "noise", "cells": int(sum(ns)), "replicas": int(sum(p.n_replicas for p in ps)),
                       "cell_updates_per_step": work,
                       "timing": "host wall clock per pass incl. table builds (tables are rebuilt every "
                                 "pass, 64 x 48 h, larger than L2) and burn counts to the host"},
            "autotuned": tuned,
            "plain": out["plain"], "batched": out["batched"],
            "batched_over_plain": out["plain"]["s_per_step"] / out["batched"]["s_per_step"],
            "tables_resident": {
                "timing": "as above, but every landscape's table is built once before the timed passes "
                          "and kept (as a served landscape's is): frontiers, ignition and burn counts only",
                "plain": out["plain_resident"], "batched": out["batched_resident"],
                "batched_over_plain": out["plain_resident"]["s_per_step"] / out["batched_resident"]["s_per_step"]}}


def serve_measure(args, sides, reqs, lands, device=0):
    """Request stream: (i) Poisson arrivals served with submit/poll (continuous
    batching), latency from arrival to counts on the host; (ii) capacity: the
    first requests all waiting at once, served vs plain (one synchronous
    c2f_simulate per request), landscapes and tables resident in both."""
    import torch
    import paper_1905_09317_gb300 as c2f
    c2f.build()
    weathers = [S.weather_stream(72, seed=600 + i) for i in range(len(sides))]
    ctx = c2f.Context(device)
    ctx.set_table_mode(not args.lazy_tables)
    ctx.set_serving(max_inflight=args.max_inflight)
    lids = [None] * len(sides)

    def params(r):
        return c2f.default_params(seed=r["seed"], n_replicas=r["n_replicas"], hours=r["hours"],
                                  ignition_mode=1, ros_sigma=0.1)

    def load(k):
        L = lands[k]
        lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
        ctx.set_weather(lid, weathers[k])
        return lid

    def stream(mode):
        for k in range(len(lids)):
            if lids[k] is not None:
                ctx.release(lids[k])
                lids[k] = None
        torch.cuda.synchronize()
        lat, work, i = [], 0, 0
        outstanding = {}
        sampler = ClockSampler(device)
        with sampler:
            t0 = time.perf_counter()
            while i < len(reqs) or outstanding:
                now = time.perf_counter() - t0
                busy = False
                while i < len(reqs) and reqs[i]["arrival_s"] <= now:
                    r = reqs[i]
                    k = r["pool_index"]
                    if lids[k] is None:
                        lids[k] = load(k)                 # a new load: inside the request's latency
                    n = lands[k].fuel.size
                    if mode == "served":
                        outstanding[ctx.submit(lids[k], params(r))] = (i, n)
                    else:                                 # plain: one synchronous call per request
                        sid = ctx.simulate(lids[k], params(r))
                        ctx.burn_prob(sid, n)
                        work += int(ctx.get_counters(sid, r["n_replicas"])[0].sum())
                        lat.append(time.perf_counter() - t0 - r["arrival_s"])
                        ctx.release(sid)
                    i += 1
                    busy = True
                if mode == "served" and outstanding:
                    for sid in [s for s in outstanding if ctx.poll(s)]:
                        j, n = outstanding.pop(sid)
                        ctx.burn_prob(sid, n)
                        work += int(ctx.get_counters(sid, reqs[j]["n_replicas"])[0].sum())
                        lat.append(time.perf_counter() - t0 - reqs[j]["arrival_s"])
                        ctx.release(sid)
                        busy = True
                if not busy:
                    nxt = reqs[i]["arrival_s"] - (time.perf_counter() - t0) if i < len(reqs) else 0.0
                    time.sleep(min(max(nxt, 0.0), 0.0005) if outstanding else max(min(nxt, 0.01), 0.0))
            wall = time.perf_counter() - t0
        lat = np.array(lat)
        return dict(wall_s=wall, requests=len(lat), cell_updates_per_s=work / wall,
                    replicas_per_s=sum(r["n_replicas"] for r in reqs) / wall,
                    p50_latency_s=float(np.percentile(lat, 50)),
                    p99_latency_s=float(np.percentile(lat, 99)),
                    mean_latency_s=float(lat.mean()), cell_updates=work, clocks=sampler.summary())

    def capacity(reqs_c):
        """the requests all waiting at t = 0, landscapes and tables resident"""
        for k in range(len(lids)):
            if lids[k] is None:
                lids[k] = load(k)
            ctx.build_ros(lids[k], c2f.default_params(hours=72, ros_sigma=0.1, ignition_mode=1), force=0)
        torch.cuda.synchronize()
        res = {}
        for mode in ("plain", "served"):
            for _ in range(2):   # the first pass warms the allocator pools; the second is timed
                work = 0
                sampler = ClockSampler(device)
                with sampler:
                    t0 = time.perf_counter()
                    if mode == "plain":
                        for r in reqs_c:
                            k = r["pool_index"]
                            sid = ctx.simulate(lids[k], params(r))
                            ctx.burn_prob(sid, lands[k].fuel.size)
                            work += int(ctx.get_counters(sid, r["n_replicas"])[0].sum())
                            ctx.release(sid)
                    else:
                        sids = [ctx.submit(lids[r["pool_index"]], params(r)) for r in reqs_c]
                        for sid, r in zip(sids, reqs_c):
                            ctx.wait(sid)
                            ctx.burn_prob(sid, lands[r["pool_index"]].fuel.size)
                            work += int(ctx.get_counters(sid, r["n_replicas"])[0].sum())
                            ctx.release(sid)
                    wall = time.perf_counter() - t0
            res[mode] = dict(wall_s=wall, cell_updates_per_s=work / wall, cell_updates=work,
                             replicas_per_s=sum(r["n_replicas"] for r in reqs_c) / wall,
                             clocks=sampler.summary())
        res["served_over_plain"] = res["plain"]["wall_s"] / res["served"]["wall_s"]
        res["requests"] = len(reqs_c)
        return res

    out = {"served": stream("served")}
    if args.serve_plain:
        out["plain_stream"] = stream("plain")
    out["capacity"] = capacity(reqs[:args.capacity_requests])
    ctx.close()
    sv = out["served"]
    return {"value": sv["cell_updates_per_s"], "unit": METRIC,
            "p50_latency_s": sv["p50_latency_s"], "p99_latency_s": sv["p99_latency_s"],
            "config": {"workload": f"Poisson arrivals {args.rate}/s for {max(r['arrival_s'] for r in reqs):.0f} s, "
                                   f"pool of {len(sides)} landscapes (sides {min(sides)}..{max(sides)}), "
                                   "replicas 32..2048, 12..72 h", "requests": len(reqs),
                       "max_inflight_epochs": args.max_inflight,
                       "timing": "host wall clock; stream: latency from arrival to burn counts on the host "
                                 "(new landscape loads inside it); capacity: the first "
                                 f"{min(len(reqs), args.capacity_requests)} requests waiting at once"},
            **out}


def large_measure(args, w, steps, device=0):
    """4096^2 cells, 72 h, 256 replicas: table build + frontier + burn counts."""
    import torch
    import paper_1905_09317_gb300 as c2f
    c2f.build()
    L = w.landscape
    n = L.fuel.size
    p = _params_of(c2f, w)
    ctx = c2f.Context(device)
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
    ctx.set_weather(lid, w.weather)
    counts = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    ctx.set_stream(stream.cuda_stream)
    ctx.set_table_mode(not args.lazy_tables)

    def step():
        ctx.build_ros(lid, p, force=2 if args.lazy_tables else 1)
        sid = ctx.simulate(lid, p)
        ctx.burn_prob_device(sid, counts.data_ptr())
        return sid

    sid = step()
    work = int(ctx.get_counters(sid, p.n_replicas)[0].sum())
    ctx.release(sid)
    fp64 = ctx.fp64_peak()
    ctx.profile(True)
    ctx.kernel_times()
    torch.cuda.synchronize()
    sampler = ClockSampler(device)
    with sampler:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            ctx.release(step())
        ev1.record(stream)
        torch.cuda.synchronize()
    dt = ev0.elapsed_time(ev1) / 1e3 / steps
    kt = ctx.kernel_times()
    ctx.close()
    roof = None if args.lazy_tables else roofline_table(kt, w, fp64)   # the table kernel dominates
    return {"value": work / dt, "unit": METRIC, "steps": steps, "ms_per_step": 1e3 * dt,
            "config": {"workload": "4096x4096 heterogeneous landscape, 72 h weather with a +90 deg wind "
                                   "shift at hour 36, 256 replicas", "cells": int(n),
                       "cell_updates_per_step": work,
                       "timing": "CUDA events on the context stream; the 87 GB table is rebuilt every step"},
            "kernel_ms_per_step": {k: v[0] / steps for k, v in kt.items()},
            "roofline": roof, "fp64_peak_gflops_measured": fp64,
            "replicas_per_s": p.n_replicas / dt, "clocks": sampler.summary()}


def run_batch(args):
    """--workload batch: the 64-landscape batch on its own line."""
    specs = S.config3_specs()
    ws = [S.config3_workload(sp) for sp in specs]
    r = batch_measure(args, ws, specs, args.steps, args.warmup)
    return {"metric": METRIC, "n_gpus": 1, "ms_per_step": 1e3 * r["batched"]["s_per_step"],
            "higher_is_better": True, "dtype": "f64", "data": "synthetic", **r,
            "cpu_baseline": _batch_cpu_baseline(args, specs)}


def _batch_cpu_baseline(args, specs):
    """The oracle beside the GPU: replica 0 of every landscape of the batch."""
    if args.no_cpu_baseline:
        return None
    procs = os.cpu_count() or 1
    rate, work, t, used = cpu_oracle_sample_rate([(("batch", i), 0) for i in range(len(specs))], procs)
    return {"value": rate, "unit": METRIC, "cores": used, "kind": "oracle",
            "sample": f"replica 0 of each of the {len(specs)} landscapes ({work} cell-updates), "
                      f"{used} single-threaded oracle processes, {t:.1f} s"}


def run_serve(args):
    """--workload serve: the request stream on its own line."""
    sides, reqs = S.serving_requests(rate=args.rate, duration_s=args.duration)
    lands = [S.heterogeneous_landscape(side, seed=500 + i) for i, side in enumerate(sides)]
    r = serve_measure(args, sides, reqs, lands)
    return {"metric": METRIC, "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": 1e3 * r["served"]["wall_s"], "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", **r}


def run_large(args):
    """--workload large: 4096^2 cells on its own line."""
    r = large_measure(args, S.config4(), args.steps)
    return {"metric": METRIC, "n_gpus": 1, "warmup": 1, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", **r, "cpu_baseline": _large_cpu_baseline(args)}


def _large_cpu_baseline(args):
    """The oracle beside the GPU: 8 of the 256 replicas (every 32nd)."""
    if args.no_cpu_baseline:
        return None
    procs = min(os.cpu_count() or 1, 8)
    rate, work, t, used = cpu_oracle_sample_rate([(("large",), r) for r in range(0, 256, 32)], procs)
    return {"value": rate, "unit": METRIC, "cores": used, "kind": "oracle",
            "sample": f"replicas 0, 32, .., 224 ({work} cell-updates), {used} single-threaded "
                      f"oracle processes, {t:.1f} s"}


def run_scenarios(args):
    """512^2 landscape, 8 weather scenarios x 24 h, 1000 replicas each drawing
    its scenario: stacked table build (K1 per scenario) + frontier + counts."""
    import torch
    import paper_1905_09317_gb300 as c2f
    c2f.build()
    w = S.config2()
    weathers, probs = S.scenario_set(8, 24)
    L = w.landscape
    n = L.fuel.size
    p = _params_of(c2f, w)
    ctx = c2f.Context(0)
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
    ctx.set_weather_scenarios(lid, weathers, probs)
    counts = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.set_stream(torch.cuda.current_stream().cuda_stream)
    ctx.set_table_mode(not args.lazy_tables)

    def step(rebuild=True):
        if rebuild:
            ctx.build_ros(lid, p, force=2 if args.lazy_tables else 1)
        sid = ctx.simulate(lid, p)
        ctx.burn_prob_device(sid, counts.data_ptr())
        return sid

    sid = step()
    work = int(ctx.get_counters(sid, p.n_replicas)[0].sum())
    drawn = np.bincount(ctx.get_scenarios(sid, p.n_replicas), minlength=len(probs))
    ctx.release(sid)
    timed = {}
    for rebuild in (True, False):
        if not rebuild:
            ctx.build_ros(lid, p, force=0)
        ctx.release(step(rebuild))
        ctx.profile(True)
        ctx.kernel_times()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.release(step(rebuild))
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        kt = ctx.kernel_times()
        ctx.profile(False)
        timed[rebuild] = (dt, {k: v[0] / args.steps for k, v in kt.items()})
    # pipelined steps, as the headline's: each step's stacked tables are built (K1,
    # context stream) while earlier steps' frontiers run on their own streams;
    # the frontier sized for one warp per SM more than a step's replicas need
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    depth = max(2, args.depth)
    ctx.set_frontier_config(32, -(-p.n_replicas // sms) + 1)
    ctx.set_serving(max_inflight=depth, max_epoch_replicas=p.n_replicas, hbm_reserve_bytes=0)

    def run_pipelined(k):
        inflight, last = [], None
        for i in range(k):
            ctx.build_ros(lid, p, force=1)
            inflight.append(ctx.submit(lid, p))
            while len(inflight) >= depth or (i == k - 1 and inflight):
                sid = inflight.pop(0)
                ctx.wait(sid)
                ctx.burn_prob_device(sid, counts.data_ptr())
                if last is not None:
                    ctx.release(last)
                last = sid
        return last

    pipelined = None
    if not args.lazy_tables:
        ctx.release(run_pipelined(depth))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        last = run_pipelined(args.steps)
        torch.cuda.synchronize()
        dt_p = (time.perf_counter() - t0) / args.steps
        assert int(ctx.get_counters(last, p.n_replicas)[0].sum()) == work, "work count changed"
        ctx.release(last)
        pipelined = {"value": work / dt_p, "unit": METRIC, "ms_per_step": 1e3 * dt_p,
                     "note": f"{depth} steps in flight: the next steps' stacked tables (K1) overlap "
                             "the current frontier (K3); host wall clock"}
    ctx.close()
    dt, kms = timed[True]
    dt_r, kms_r = timed[False]
    return {"metric": METRIC, "value": work / dt, "unit": METRIC, "n_gpus": 1, "steps": args.steps,
            "warmup": 2, "ms_per_step": 1e3 * dt, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "512x512 heterogeneous landscape, 8 weather scenarios x 24 h "
                                   "(weights 1,2,3,4,4,3,2,1), 1000 replicas drawing their scenario, "
                                   "random ignitions, lognormal(0,0.1) ROS noise",
                       "tables": "lazy" if args.lazy_tables else "eager",
                       "cell_updates_per_step": work,
                       "replicas_per_scenario": drawn.tolist()},
            "kernel_ms_per_step": kms, "replicas_per_s": p.n_replicas / dt,
            "tables_reused": {"value": work / dt_r, "unit": METRIC, "ms_per_step": 1e3 * dt_r,
                              "kernel_ms_per_step": kms_r,
                              "note": "the 8 stacked tables built once; each step K2 + K3 + K4"},
            "pipelined": pipelined}


def run_burnhours(args):
    """512^2 landscape, 48 h weather, 1000 replicas whose fires burn only the first B
    hours of each day, B drawn per replica from {6..12} (A5, condition (1)), against
    the same replicas with no limit.  A step: table (K1) + K2 + K3 + K4, one at a time."""
    import torch
    import paper_1905_09317_gb300 as c2f
    c2f.build()
    w = S.config2(hours=48)
    L = w.landscape
    n = L.fuel.size
    ctx = c2f.Context(0)
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
    ctx.set_weather(lid, w.weather)
    counts = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.set_stream(torch.cuda.current_stream().cuda_stream)
    out = {}
    for name, over in (("limited", dict(burn_hours_min=6, burn_hours_max=12)), ("unlimited", {})):
        p = _params_of(c2f, w, **over)

        def step():
            ctx.build_ros(lid, p, force=1)
            sid = ctx.simulate(lid, p)
            ctx.burn_prob_device(sid, counts.data_ptr())
            return sid

        sid = step()
        work = int(ctx.get_counters(sid, p.n_replicas)[0].sum())
        ctx.release(sid)
        ctx.profile(True)
        ctx.kernel_times()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.release(step())
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        kt = ctx.kernel_times()
        ctx.profile(False)
        out[name] = {"value": work / dt, "unit": METRIC, "ms_per_step": 1e3 * dt, "cell_updates_per_step": work,
                     "kernel_ms_per_step": {k: v[0] / args.steps for k, v in kt.items()}}
    ctx.close()
    lim = out["limited"]
    return {"metric": METRIC, "value": lim["value"], "unit": METRIC, "n_gpus": 1, "steps": args.steps,
            "warmup": 1, "ms_per_step": lim["ms_per_step"], "higher_is_better": True, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "512x512 heterogeneous landscape, 48 h hourly weather, 1000 replicas "
                                   "burning the first B hours of each day, B uniform in {6..12} per "
                                   "replica, random ignitions, lognormal(0,0.1) ROS noise",
                       "timing": "host wall clock, one step at a time (table rebuilt every step)"},
            "limited": lim, "unlimited": out["unlimited"]}


def run_replica_profile(args):
    """The 512^2 x 1000-replica frontier, one launch alone with the per-replica
    counters on (the profiling build of the kernel): where a visited period's
    cycles go, averaged over every visited period of every replica."""
    import paper_1905_09317_gb300 as c2f
    c2f.build()
    w = S.config2(n_replicas=args.replicas)
    L = w.landscape
    p = _params_of(c2f, w)
    R = p.n_replicas
    with c2f.Context(0) as ctx:
        lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
        ctx.set_weather(lid, w.weather)
        ctx.release(ctx.simulate(lid, p))                       # tables built, warm-up
        ctx.profile(True, replicas=True)
        sid = ctx.simulate(lid, p)
        pr = ctx.replica_profile(sid, R).astype(np.float64)
        ctx.profile(False)
        ctx.release(sid)
    total, bound, send, new, periods, hits, newc, longest, walk, comp, rounds, newit = pr[:, :12].T
    v = periods.sum()
    per = lambda x: float(x.sum() / v)   # noqa: E731
    return {"workload": WORKLOAD, "replicas": R, "counters": "c2f_get_replica_profile, profiling build",
            "visited_periods_per_replica": float(periods.mean()),
            "cycles_per_visited_period": {"all": per(total), "hour_boundary": per(bound),
                                          "calendar_walk": per(walk), "crossing_rounds": per(send - walk),
                                          "new_cell_setup": per(new)},
            "per_visited_period": {"crossing_cells": per(hits), "rounds": per(rounds), "new_cells": per(newc),
                                   "setup_passes": per(newit)},
            "setup_pass_cycles": float(new.sum() / max(newit.sum(), 1)),
            "replica_cycles": {"median": float(np.median(total)), "max": float(total.max())},
            "longest_list_median": float(np.median(longest)), "compactions": float(comp.sum())}


def run_compare(args):
    """Sec. 4.1 scar comparison: the 512^2 workload run with Eq. (1) and with the
    centre-offset ellipse ray (1000 replicas each, ignition steps kept), then
    hourly MSE / SSIM and the final scars' norm for every replica pair."""
    import torch
    import paper_1905_09317_gb300 as c2f
    c2f.build()
    w = S.config2()
    L = w.landscape
    n = L.fuel.size
    R, H = w.params["n_replicas"], w.params["hours"]
    ctx = c2f.Context(0)
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
    ctx.set_weather(lid, w.weather)
    out = c2f.OUT_SCARS | c2f.OUT_COUNTERS | c2f.OUT_IGN_STEPS
    sx = ctx.simulate(lid, _params_of(c2f, w, ellipse_mode=0, outputs=out))
    sy = ctx.simulate(lid, _params_of(c2f, w, ellipse_mode=1, outputs=out))
    stream = torch.cuda.Stream()   # a real stream (the default one would read as NULL)
    ctx.set_stream(stream.cuda_stream)
    mse = torch.empty(R * H, dtype=torch.float64, device="cuda")
    ssim = torch.empty(R * H, dtype=torch.float64, device="cuda")
    dn = torch.empty(R, dtype=torch.float64, device="cuda")

    def step():
        ctx.compare_scars_device(sx, sy, mse.data_ptr(), ssim.data_ptr(), dn.data_ptr())

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    m = mse.view(R, H).cpu().numpy()
    q = ssim.view(R, H).cpu().numpy()
    ctx.close()
    # algorithmic bytes of the launch: both runs' ignition steps read once, the
    # metrics written once (the final norm comes from the last hour's counts)
    by = 2 * R * n * 4 + R * H * 16 + R * 8
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    ach = by / (ms / 1e3) / 1e9
    return {"metric": "replica-pairs/s", "value": R / (ms / 1e3), "unit": "replica-pairs/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "512x512 heterogeneous landscape, 24 h, 1000 replicas run with Eq. (1) "
                                   "and with the centre-offset ellipse ray; hourly MSE and SSIM and the "
                                   "final scars' norm per replica pair (Sec. 4.1)",
                       "inputs": "2.1 GB of ignition steps, larger than L2"},
            "roofline": {"kernel": "k_compare_hours", "bound": "hbm", "achieved": ach,
                         "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": None,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
            "result": {"mse_final_mean": float(m[:, -1].mean()), "ssim_final_mean": float(q[:, -1].mean()),
                       "mse_hour1_mean": float(m[:, 0].mean()), "ssim_hour1_mean": float(q[:, 0].mean())}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--replicas", type=int, default=1000,
                    help="replicas per GPU (the workload has 1000; fewer only for profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--frontier-threads", type=int, default=0,
                    help="frontier CTA size (64/128/256); 0 = library default")
    ap.add_argument("--smem-plane-bytes", type=int, default=1, help="0 = frontier state in global memory")
    ap.add_argument("--cpu-sample", type=int, default=1000)
    ap.add_argument("--ref-sample", type=int, default=128)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lazy-tables", action="store_true",
                    help="ROS-table rows computed on demand inside the frontier instead of by K1")
    ap.add_argument("--depth", type=int, default=3, help="pipelined steps in flight (>= 2)")
    ap.add_argument("--serial", action="store_true",
                    help="one synchronous step at a time (no overlap of K1 with the previous frontier)")
    ap.add_argument("--workload", default="landscape",
                    choices=["landscape", "batch", "serve", "large", "scenarios", "compare", "burnhours",
                             "replica-profile"])
    ap.add_argument("--tune-sample", type=int, default=4096, help="batch: autotuner replica sample")
    ap.add_argument("--rate", type=float, default=50.0, help="serve: arrivals per second")
    ap.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    ap.add_argument("--max-inflight", type=int, default=3, help="serve: concurrent epochs")
    ap.add_argument("--serve-plain", action="store_true",
                    help="serve: also replay the stream with one synchronous call per request")
    ap.add_argument("--serve-window", type=float, default=10.0,
                    help="default line: seconds of Poisson arrivals in its request-stream section")
    ap.add_argument("--capacity-requests", type=int, default=200,
                    help="request stream: requests waiting at once in the capacity comparison")
    ap.add_argument("--plain-steps", type=int, default=10,
                    help="default line: steps of the plain (one synchronous call per step) timing")
    ap.add_argument("--no-extras", action="store_true",
                    help="default line without its batch, request-stream and 4096^2 sections")
    ap.add_argument("--trace-steps", type=int, default=8,
                    help="pipelined steps under the launch trace after the timed regions (0: none)")
    ap.add_argument("--trace-out", default=None, help="write the launch-trace summary to this file")
    args = ap.parse_args()
    world_env = int(os.environ.get("WORLD_SIZE", "1"))
    err = gpus_mismatch(args.gpus, world_env)
    if err:
        print(err, file=sys.stderr, flush=True)
        sys.exit(2)
    if args.workload != "landscape" and args.impl == "ours":
        fn = {"batch": run_batch, "serve": run_serve, "large": run_large,
              "scenarios": run_scenarios, "compare": run_compare, "burnhours": run_burnhours,
              "replica-profile": run_replica_profile}[args.workload]
        print(json.dumps(fn(args)), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    out = run_ours(args, rank, world, local_rank)
    if out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
