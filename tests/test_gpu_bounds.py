"""Bounds-checked build (-DPF_BOUNDS_CHECK; compute-sanitizer stands in for
nothing here): every global and shared-memory index of the kernels passes a
checker that counts and neutralises out-of-range indices.  The battery in
bounds_battery.py runs tiny, odd and ragged grids through every scheme,
precision and variant against the checked library; no index may fail."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_has_no_out_of_range_index():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12448_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, PF_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_battery.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["checked"] and out["cases"] >= 150, out
    assert out["failures"] == 0, out
