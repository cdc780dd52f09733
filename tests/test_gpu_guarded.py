"""The guarded build (index checks in the plane path's kernels, see
sgm_debug_guard_hits in sgm.h) over shapes that reach every edge of the
kernels' indexing: results equal the oracle's and no index leaves its buffer.
An out-of-range read that happens not to change a result would pass the
parity tests; here it would be counted."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_guarded_build_stays_in_bounds_and_matches_the_oracle():
    from paper_1807_06271_gb300 import build
    lib = build.build(guarded=True)
    env = dict(os.environ, SGM_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "guarded_run.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["library"] == "libsgm_guarded.so"
    assert out["mismatches"] == []
    assert out["hits"] == 0
