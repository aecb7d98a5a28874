"""The bounds-checked build (libalb_checked.so) is itself exact and clean.

Every index the round kernels use is tested in that build; an out-of-range one is skipped and
recorded instead of being accessed. A child process loads it (ALB_CHECKED=1), runs every
application, the batched calls and the allocation-free BFS on small graphs under several
load-balancing settings, compares each result with the CPU oracle and requires every handle's
record to stay zero (tests/checked_parity.py).
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_matches_the_oracle_with_no_bounds_failure():
    from paper_1911_09135_gb300 import _build
    _build.build_alb(checked=True)  # no-op when current
    env = dict(os.environ, ALB_CHECKED="1")
    proc = subprocess.run([sys.executable, "-m", "tests.checked_parity"], cwd=ROOT, env=env,
                          stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=900)
    assert proc.returncode == 0, proc.stdout[-4000:]
    assert "CHECKED PARITY OK" in proc.stdout, proc.stdout[-4000:]
