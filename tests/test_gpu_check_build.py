"""The bounds-checking build (liblpp_check.so, compiled with -DLPP_CHECK): every hot kernel
checks its data-dependent indices (sorted-particle positions, tile coordinates and range
counts, scatter cells, pencil and column offsets of the passes, mode-pair offsets of the
combine, the coefficient permutation) and records a violation as LPP_ERR_BOUNDS instead of
making the access.  The parity cases run through it in a child process (LPP_CHECK=1 selects
the library at load time) and must pass with no violation recorded.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checking_build_runs_the_parity_cases_clean():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2202_11839_gb300 import build as B
    B.build(check=True)
    env = dict(os.environ, LPP_CHECK="1")
    cmd = [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_gpu_parity.py"), "-q", "-x",
           "-p", "no:cacheprovider", "-k", "fp64_parity or fp32_parity or host_inputs"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
    # the child loaded the checking build
    code = "from paper_2202_11839_gb300 import lpp as L; print(L.LIB_PATH)"
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True)
    assert out.stdout.strip().endswith("liblpp_check.so"), out.stdout
