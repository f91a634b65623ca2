"""The index-checked build (MC_CHECKED: every table, pixel, radial-bin, voxel,
majorant-cell and hat index is checked at run time, a bad one reported as
MC_EFLAG_BOUNDS and clamped) runs the walk in all phase functions and image
modes, the delta-tracking walk, the density gradient and the homogeneous
adjoint without a single report, and its results equal the normal build's
bit for bit (integer tallies) or to the last bits of the double sums
(gradients, whose atomics run in another order)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(out, checked):
    env = dict(os.environ)
    env.pop("MC_CHECKED", None)
    if checked:
        env["MC_CHECKED"] = "1"
    p = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_workloads.py"), out], env=env,
                       capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    return np.load(out)


def test_checked_build_reports_nothing_and_matches(tmp_path):
    from paper_2507_23189_gb300 import build
    build.build()
    build.build_checked()
    a = _run(str(tmp_path / "normal.npz"), False)
    b = _run(str(tmp_path / "checked.npz"), True)
    for k in a.files:
        if k.endswith("_err"):
            assert int(b[k]) == 0, (k, int(b[k]))      # no index check fired
            assert int(a[k]) == 0, (k, int(a[k]))
        elif k in ("gadj_grad", "gadj_val", "adj"):
            np.testing.assert_allclose(b[k], a[k], rtol=1e-6, atol=1e-6 * float(np.max(np.abs(a[k]))))
        else:
            np.testing.assert_array_equal(b[k], a[k], err_msg=k)
