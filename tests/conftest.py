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


def oracle_parallel(aut, text, lo=0, hi=None, parts=0):
    """The oracle's match set for the starts in [lo, hi) of `text`, cut into
    start windows scanned by one host thread each (lazy data partitioning,
    Sec. III.D.2: a window's instances read on past its end). The C oracle
    releases the interpreter lock, so the windows run on every host core."""
    import concurrent.futures
    import numpy as np
    import oracle
    hi = len(text) if hi is None else hi
    cores = max(1, os.cpu_count() or 1)
    k = max(1, parts or 4 * cores)
    bounds = [lo + (hi - lo) * i // k for i in range(k + 1)]
    with concurrent.futures.ThreadPoolExecutor(max_workers=cores) as ex:
        got = list(ex.map(lambda i: oracle.scan(aut, text, bounds[i], bounds[i + 1]), range(k)))
    got = [g for g in got if len(g)]
    if not got:
        return np.zeros((0, 3), dtype=np.uint32)
    return oracle.sort_matches(np.concatenate(got))
