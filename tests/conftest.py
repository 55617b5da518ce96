import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size inputs")


def read_golden(name):
    """Rows (label, start, end) of a fixture under tests/golden/ plus its input."""
    path = os.path.join(ROOT, "tests", "golden", name)
    rows, text = [], None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line.startswith("# input:"):
                text = line.split(":", 1)[1].strip()
            if not line or line.startswith("#"):
                continue
            lab, i, j = line.rsplit(" ", 2)
            rows.append((lab, int(i), int(j)))
    return text, sorted(rows)
