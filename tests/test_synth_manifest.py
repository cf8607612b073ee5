"""The seeded synthetic inputs are the ones recorded in
tests/golden/synth_manifest.json (written by make_synth_manifest.py beside
it): every workload's landscape arrays, weather and parameters, the batch
specs and three of its landscapes, the weather scenarios and the request
stream.  Checksums are of the generating machine's numpy, whose float
transcendentals (Horn's aspect, fBm) may differ in the last bit elsewhere, so
the comparison runs on the same machine type only."""
import importlib.util
import json
import os
import platform

import pytest

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_synthetic_inputs_match_the_manifest():
    with open(os.path.join(GOLD, "synth_manifest.json")) as f:
        want = json.load(f)
    if platform.machine() != want["machine"]:
        pytest.skip(f"manifest written on {want['machine']}")
    spec = importlib.util.spec_from_file_location("make_synth_manifest", os.path.join(GOLD, "make_synth_manifest.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    got = json.loads(json.dumps(mod.build(), sort_keys=True))
    for key in want:
        assert got[key] == want[key], key
