"""The bounds-checked build (the library compiled with CSG_CHECKED, standing in for a memory
checker): every guarded access the kernels compute stays inside its buffer on small and
odd-sized sets, a mixed batch, a caller's bitmap, the allocation-free call, the service and
the bench-size set, and the results equal the oracle's.  The checked library is built here
and run in a separate process, so the binding loads it instead of the normal one."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_runs_clean():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_03013_gb300 import _build
    lib = _build.build(checked=True)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_workloads.py"), lib],
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "checked build clean" in r.stdout
