import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU check")


def read_golden_grid(name):
    """Parse a golden text fixture: '#' comments, 'key: value' scalars, then grid rows."""
    path = os.path.join(ROOT, "tests", "golden", name)
    meta, grid = {}, []
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if ":" in line:
                k, v = line.split(":", 1)
                meta[k.strip()] = v.strip()
            else:
                grid.append([int(t) for t in line.split()])
    return meta, grid
