"""The bounds-checked build (-DPP_CHECKED): every particle-kernel index into
the mesh or the shared-memory windows is tested against its array.  On the
cases of tests/checked_cases.py (the tiled kernel with its drift fallback, the
FP64 global kernels for every shape, the direct current, the 4th-order step,
walls with an open end, an injector and a sliding window)
it must report no violation and give the normal build's fields."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_finds_no_out_of_bounds_index():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_4575_gb300 import build
    build.build()
    build.build(checked=True)   # several minutes: the checks are inlined at every access
    from tests import checked_cases
    plain = checked_cases.run_cases()
    env = dict(os.environ, PP_GB300_CHECKED="1")
    r = subprocess.run([sys.executable, "-m", "tests.checked_cases", ROOT], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    checked = json.loads(r.stdout.strip().splitlines()[-1])
    assert set(checked) == set(plain)
    for name, (status, fields) in checked.items():
        assert status == 0, (name, status)          # PP_EBOUNDS would be 10
        a, b = np.asarray(fields), np.asarray(plain[name][1])
        tol = 1e-12 if name.startswith("fp64") else 1e-4
        assert np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1e-30), name
