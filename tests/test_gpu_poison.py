"""Uninitialised-memory check: the GPU suites again with poisoned allocations.

With DPP_POISON_ALLOC=1 the library fills every buffer it allocates with 0xFF
bytes (NaN for FP64/FP32, -1 for integers) before first use. Any kernel that
reads memory the library never wrote then turns results into NaN or wrong
indices, which the oracle comparisons catch. The variable is read once per
process, so the suites run in a child pytest process.
"""
import os
import subprocess
import sys

import pytest

from gpu_helpers import needs_gpu

pytestmark = [pytest.mark.gpu, needs_gpu]

HERE = os.path.dirname(os.path.abspath(__file__))


def test_suites_pass_with_poisoned_allocations():
    env = dict(os.environ, DPP_POISON_ALLOC="1")
    targets = [os.path.join(HERE, f) for f in
               ("test_gpu_parity.py", "test_gpu_mixed.py", "test_gpu_batched.py",
                "test_gpu_adjoint.py", "test_gpu_sell.py", "test_gpu_scale_split.py",
                "test_gpu_matfree.py", "test_gpu_inner.py", "test_gpu_q1.py", "test_gpu_edge.py")]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-m", "gpu", "-p", "no:cacheprovider",
                        *targets], env=env, cwd=os.path.dirname(HERE), capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
