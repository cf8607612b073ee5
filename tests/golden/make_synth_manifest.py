"""Writes synth_manifest.json beside this file: sha256 checksums of the seeded
synthetic inputs (c2f_synth) that the tests and the benchmark generate --
the five workloads' landscapes, weather and parameters, the batch's 64
landscape specs and three of its landscapes, the weather-scenario set and the
request stream -- so that a change to the generator cannot pass unnoticed.
Run from the repository root on an x86-64 host:

    python tests/golden/make_synth_manifest.py
"""
import json
import os
import platform
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import c2f_synth as S  # noqa: E402


def build():
    specs = S.config3_specs()
    by_side = sorted(range(len(specs)), key=lambda i: specs[i]["side"])
    picks = [by_side[0], by_side[len(by_side) // 2], by_side[-1]]
    weathers, weights = S.scenario_set()
    sides, reqs = S.serving_requests()
    out = {
        "machine": platform.machine(),
        "config1": S.workload_digest(S.config1()),
        "config2": S.workload_digest(S.config2()),
        "config3_specs": S.digest(json.dumps(specs, sort_keys=True).encode()),
        "config3_landscapes": {str(i): S.workload_digest(S.config3_workload(specs[i])) for i in picks},
        "config4": S.workload_digest(S.config4()),
        "scenario_set": S.digest(weathers, weights),
        "serving_requests": S.digest(json.dumps([sides, reqs], sort_keys=True).encode()),
        "n_requests": len(reqs),
    }
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "synth_manifest.json")
    with open(path, "w") as f:
        json.dump(build(), f, indent=1, sort_keys=True)
        f.write("\n")
    print("wrote", path)
