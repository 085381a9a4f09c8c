"""A bounds-checked build (LBM_BOUNDS_CHECK=1: every population, psi and psi-ring access of the step
kernels checked against its array, an access outside counted and redirected) runs the cases of
tests/bounds_cases.py -- periodic, one-pass, FP16, walls at the z ends, a solid cylinder, a batch,
degenerate extents and an axis at the maximum extent, on both lattices -- with no access outside
its arrays, and to the same final populations as the normal build."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _run(lib):
    env = dict(os.environ, LBM_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py")], capture_output=True, text=True,
                       env=env, cwd=ROOT, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_bounds_checked_build(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2306_16274_gb300 import build as B
    checked = B.build_variant(str(tmp_path / "checked"), ["-DLBM_BOUNDS_CHECK=1"])
    normal = _run(B.LIB)
    debug = _run(checked)
    assert normal["violations"] == 0
    assert debug["violations"] == 0
    assert debug["digests"] == normal["digests"]
