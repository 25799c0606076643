import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def load_golden(name):
    """Parse a tests/golden/*.txt fixture: '[key]' headers followed by rows of ints."""
    path = os.path.join(ROOT, "tests", "golden", name)
    out, key = {}, None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                key = line.strip("[]")
                out[key] = []
                continue
            out[key].append([int(t) for t in line.split()])
    return out
