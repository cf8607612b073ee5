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
