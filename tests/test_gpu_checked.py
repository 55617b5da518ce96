"""The parity suite against the checked build (libpfsm_checked.so, device
code compiled with PFSM_CHECKED: every data-dependent table, record, list,
queue and staging index is tested before use, and a failure is reported as
PFSM_E_CHECK instead of trapping). The GPU parity files run in a child
process with PFSM_CHECKED=1, which makes the binding load that build; they
must pass unchanged, which also shows that no check fires on them."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suite_under_the_checked_build():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_1716_gb300 import build
    path = build.build(checked=True)
    assert path.endswith("libpfsm_checked.so") and os.path.exists(path)
    env = dict(os.environ, PFSM_CHECKED="1")
    probe = subprocess.run(
        [sys.executable, "-c", "import paper_1110_1716_gb300 as P; P.load_library(); print(P.LIB_PATH)"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert probe.returncode == 0, probe.stderr[-2000:]
    assert probe.stdout.strip().endswith("libpfsm_checked.so")
    files = ["tests/test_gpu_scan.py", "tests/test_gpu_batch.py", "tests/test_gpu_eps.py",
             "tests/test_gpu_union.py", "tests/test_gpu_unaligned.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu and not slow",
                        "-p", "no:cacheprovider", *files],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
