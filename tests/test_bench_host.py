"""Host-side pieces of the benchmark (no GPU): the sampled oracle timing that
stands beside the GPU numbers of the batch and 4096^2 workloads, and the
reference arm's JSON line."""
import json
import os
import subprocess
import sys

import numpy as np

import bench
import c2f_synth as S
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_sampled_oracle_rate_counts_the_replicas_it_ran():
    specs = S.config3_specs()
    i = int(np.argmin([sp["side"] for sp in specs]))      # the smallest batch landscape
    rate, work, t, used = bench.cpu_oracle_sample_rate([(("batch", i), 0), (("batch", i), 1)], 2)
    w = S.config3_workload(specs[i])
    L = w.landscape
    o = oracle.Oracle(L.fuel, L.slope, L.aspect, cell_size=L.cell_size, weather=w.weather, **w.params)
    assert work == o.run_replica(0)["work"] + o.run_replica(1)["work"]
    assert used == 2 and t > 0 and rate == work / t


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--ref-sample", "4"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    d = json.loads(lines[-1])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_gpus_must_match_the_launched_processes():
    """--gpus N with N processes launched is accepted; anything else is refused
    before any device work, so that a line never claims GPUs it did not time."""
    assert bench.gpus_mismatch(1, 1) is None and bench.gpus_mismatch(8, 8) is None
    assert bench.gpus_mismatch(2, 1) and bench.gpus_mismatch(1, 4) and bench.gpus_mismatch(0, 1)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--steps", "1"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT,
                         env={k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK")})
    assert out.returncode == 2 and "--gpus 2" in out.stderr and not out.stdout.strip()


def test_timeline_summary_of_trace_records():
    """bench.timeline on hand-made c2f_trace records: two builds of 2 CTAs on a
    2-SM device, each followed by a simulation of two replicas."""
    ms = 1_000_000   # ns

    def rec(kind, sm, aux, tag, t0, t1):
        return [kind | (sm << 8) | (aux << 32), tag, int(t0 * ms), int(t1 * ms)]

    r = np.array([
        rec(1, 0, 0, 1, 0.0, 2.0), rec(1, 1, 0, 1, 0.0, 1.0),          # build 1: 0..2 ms, 3 CTA-ms
        rec(2, 0, 0, 1, 2.0, 5.0), rec(2, 1, 1, 1, 2.0, 4.0),          # sim 1 replicas: 3 and 2 ms
        rec(1, 0, 0, 2, 3.0, 4.0), rec(1, 1, 0, 2, 3.0, 4.0),          # build 2: 3..4 ms, 2 CTA-ms
        rec(2, 0, 0, 2, 4.0, 8.0), rec(2, 1, 1, 2, 4.0, 5.0),          # sim 2 replicas: 4 and 1 ms
    ], dtype=np.uint64)
    out, lines = bench.timeline(r, sms=2)
    assert out["builds"] == 2 and out["simulations"] == 2
    assert out["k1_ms"] == 1.5                                         # median of spans 2 and 1
    assert abs(out["k1_ctas_per_sm"] - (3 + 2) / (2 + 1) / 2) < 1e-12
    assert out["k1_gap_ms"] == 1.0 and out["build_period_ms"] == 3.0
    # replica time inside the build windows: build 2 (3..4 ms) overlaps both of sim 1's
    # replicas (2..5 and 2..4 ms) for 1 ms each; build 1 (0..2 ms) overlaps none
    assert abs(out["replicas_per_sm_during_k1"] - 2.0 / 3.0 / 2) < 1e-12
    assert out["replica_ms_median"] == 2.5 and out["replica_ms_max"] == 4.0
    assert out["frontier_span_ms"] == 3.5                              # spans 3 and 4
    assert len(lines) == 4 and lines[0].startswith("K1 build")


def test_frontier_roofline_entry_follows_its_inputs():
    """The K3 roofline entry from a launch time: every figure is the profile's
    per-replica or per-update constant scaled by the workload and divided by
    the same duration; none of the measured fractions exceeds 1."""
    w = S.config2()
    work = 219342267
    r = bench.frontier_roofline({"frontier": (44.0, 10)}, w, work, {"hbm_gbs": 6800.0}, 152, 2070.0)
    s = 4.4e-3
    R = w.params["n_replicas"]
    assert r["bound"] == "latency" and abs(r["ms_per_launch"] - 4.4) < 1e-12
    assert abs(r["traffic"] - bench.FRONTIER_DRAM_BYTES_PER_REPLICA * R) < 1
    assert abs(r["achieved"] - r["traffic"] / s / 1e9) < 1e-9 and 0 < r["frac"] < 1
    inst = bench.FRONTIER_WARP_INST_PER_UPDATE * work
    assert abs(r["issue"]["warp_inst_per_launch"] - inst) < 1
    assert abs(r["issue"]["frac"] - inst / s / (152 * 4 * 2070e6)) < 1e-12 and r["issue"]["frac"] < 1
    assert abs(r["l2"]["achieved_gbs"] - bench.FRONTIER_L2_BYTES_PER_REPLICA * R / s / 1e9) < 1e-9
    assert abs(r["period_method_equiv_gbs"] - 194.0 * work / s / 1e9) < 1e-6
    assert bench.frontier_roofline({"frontier": (0.0, 0)}, w, work, {}, 152, 2070.0) is None
