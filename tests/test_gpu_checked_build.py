"""The checked build (libptycho_checked.so: index checks in the kernels at
the shared-memory slot function, the window coordinates of every pointwise
stage operation and the item indices, reported by ptycho_check as
PTYCHO_ECHECK) runs every window size, the tensor-core tile, the work
queue, a skipped position and fused steps without a failed check, and gives
the results of the normal build.  It runs in a child process, since one
process loads one build of the library."""
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import rel_l2

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CHILD = os.path.join(HERE, "checked_build_run.py")
LIB_CHECKED = os.path.join(os.path.dirname(HERE), "paper_2505_14372_b300", "libptycho_checked.so")


def _run(tmp_path, which):
    out = tmp_path / f"{which}.npz"
    env = dict(os.environ)
    env["PTYCHO_LIBRARY"] = which
    r = subprocess.run([sys.executable, CHILD, str(out)], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return dict(np.load(out))


def test_checked_build_passes_its_checks_and_matches_the_normal_build(tmp_path):
    if not os.path.exists(LIB_CHECKED):
        pytest.fail("libptycho_checked.so is missing: python -m paper_2505_14372_b300.build --checked")
    chk = _run(tmp_path, "checked")  # ECHECK from any ptycho_check would fail the child
    ref = _run(tmp_path, "normal")
    assert int(chk["checked"]) == 1 and int(ref["checked"]) == 0
    # the skipped position is reported as out of bounds, not as an index error
    assert int(chk["oob_code"]) == -2 and int(ref["oob_code"]) == -2
    for k in ref:
        if k in ("checked", "oob_code"):
            continue
        a, b = chk[k], ref[k]
        if a.ndim == 0 or k == "step_stats":
            assert np.allclose(a, b, rtol=1e-5, atol=0), (k, a, b)
        else:
            assert rel_l2(a, b) < 1e-5, (k, rel_l2(a, b))
