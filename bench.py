"""Benchmark: Monte-Carlo fire growth on one GB300 (or N, replica-sharded).

Workload (one "step" = one pass of the whole path): the 512x512 heterogeneous
landscape, 24 h hourly weather, 1000 replicas with random ignitions and
lognormal(0, 0.1) ROS noise -- ROS table (K1), ignition (K2), frontier (K3)
and burn-probability counts (K4).  Metric: cell-updates/s, the number of
(burning cell, fire period) pairs of Algorithm 1 per second, summed over
replicas; replicas/s is reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own 1000 replicas (replica ids offset by
rank), so per-GPU work is fixed (weak scaling) and no collective touches the
data path; the timing is max-over-ranks.
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

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
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
        for ln in self.lines:
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


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1905_09317_gb300 as c2f

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c2f.build()
    w = S.config2(n_replicas=args.replicas)
    L = w.landscape
    n = L.fuel.size
    R = w.params["n_replicas"]
    keys = {f[0] for f in c2f.SimParams._fields_}
    params = c2f.default_params(**{k: v for k, v in w.params.items() if k in keys})
    params.seed = params.seed + 7919 * rank          # each rank: its own replicas

    ctx = c2f.Context(local_rank)
    if args.frontier_threads:
        ctx.set_frontier_config(args.frontier_threads, args.smem_plane_bytes)
    stream = torch.cuda.current_stream(dev)
    ctx.set_stream(stream.cuda_stream)
    lid = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
    ctx.set_weather(lid, w.weather)
    counts_dev = torch.empty(n, dtype=torch.int32, device=dev)

    def step():
        ctx.build_ros(lid, params, force=True)                  # a1 + a2 (K1)
        sid = ctx.simulate(lid, params)                         # a3..a8 (K2, K3)
        ctx.burn_prob_device(sid, counts_dev.data_ptr())        # a9 (K4)
        return sid

    # warm-up (also fixes the deterministic work count of the step)
    for _ in range(max(args.warmup, 0)):
        sid = step()
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
        sids = []
        for _ in range(args.steps):
            sids.append(step())
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    kt = ctx.kernel_times()
    ctx.profile(False)
    last_work, _, _ = ctx.get_counters(sids[-1], R)
    assert int(last_work.sum()) == work_per_step, "work count changed between steps"
    for s in sids:
        ctx.release(s)

    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(t.item())

    # e2e: host buffers through the C ABI, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        host_counts = np.empty(n, dtype=np.uint32)
        h2d = L.fuel.nbytes + L.slope.nbytes + L.aspect.nbytes + w.weather.nbytes
        e2e_steps = max(1, min(args.steps, 3))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            l2 = ctx.load_landscape(L.fuel, L.slope, L.aspect, cell_size=L.cell_size)
            ctx.set_weather(l2, w.weather)
            s2 = ctx.simulate(l2, params)
            host_counts[:] = ctx.burn_prob(s2, n)
            ctx.release(s2)
            ctx.release(l2)
        torch.cuda.synchronize(dev)
        e2e_s = time.perf_counter() - t0
        te = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        if world > 1:
            torch.distributed.all_reduce(te, op=torch.distributed.ReduceOp.MAX)
        e2e = dict(value=work_per_step * world * e2e_steps / float(te.item()), unit=METRIC,
                   h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(host_counts.nbytes),
                   steps=e2e_steps)

    out = None
    if rank == 0:
        total_work = work_per_step * world * args.steps
        value = total_work / (ms_max / 1e3)
        peaks = measured_peaks()
        fam = {k: v for k, v in kt.items()}
        dom = max(fam, key=lambda k: fam[k][0])
        roof = roofline(dom, fam, w, work_per_step, peaks)
        launches = int(sum(v[1] for v in fam.values())) + 1 * args.steps   # + hour prep per K1
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
                       "parallelism": f"replica-sharded x{world}"},
            "replicas_per_s": R * world * args.steps / (ms_max / 1e3),
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in fam.items()},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": sampler.summary(),
        }
    ctx.release(lid)
    ctx.close()
    return out


def roofline(dom, fam, w, work_per_step, peaks):
    """Roofline entry of the dominant kernel family (algorithmic bytes / flops per launch)."""
    ms, launches = fam[dom]
    if launches == 0:
        return None
    n = w.landscape.fuel.size
    H = w.params["hours"]
    hbm = peaks.get("hbm_gbs", 6800.0)
    per_launch_s = ms / launches / 1e3
    if dom == "ros_table":
        # FP64-ALU bound: binary64 operations per cell-hour
        flops = FP64_OPS_PER_CELL_HOUR * n * H
        peak = FP64_PEAK_GFLOPS
        ach = flops / per_launch_s / 1e9
        return {"kernel": "k_ros_table", "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "GFLOP/s (fp64)", "frac": ach / peak, "traffic": None,
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x SM clock"}
    if dom == "frontier":
        by = FRONTIER_BYTES_PER_UPDATE * work_per_step
        ach = by / per_launch_s / 1e9
        return {"kernel": "k_frontier", "bound": "hbm", "achieved": ach, "peak": hbm,
                "unit": "GB/s", "frac": ach / hbm, "traffic": None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    by = w.params["n_replicas"] * ((w.landscape.fuel.shape[1] + 31) // 32) * 4 * \
        w.landscape.fuel.shape[0] + 4 * n
    ach = by / per_launch_s / 1e9
    return {"kernel": "k_" + dom, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm, "traffic": None}


# algorithmic figures (the design doc states how they are derived)
FRONTIER_BYTES_PER_UPDATE = 194.0
FP64_OPS_PER_CELL_HOUR = 700.0
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
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
    args = ap.parse_args()
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
