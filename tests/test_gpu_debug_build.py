"""The debug build (XYL_DEBUG): kernels check every neighbour id, row length
and colour-class bound before following it.  It must compute exactly what the
release build computes, and turn an out-of-range id in the device CSR into the
status XYL_EBOUNDS instead of an access outside its array.

The debug library is built on demand (a second copy of the library) and runs
in a child process with XYL_DEBUG=1; the release run uses the same case list
in this process (tests/debug_build_child.py)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CHILD = os.path.join(HERE, "debug_build_child.py")


@pytest.fixture(scope="module")
def debug_lib():
    from paper_1211_3991_gb300 import build
    return build.build(debug=True)


def _run_child(out, corrupt):
    env = dict(os.environ, XYL_DEBUG="1")
    subprocess.run([sys.executable, CHILD, str(out), "true" if corrupt else "false"], env=env, check=True,
                   timeout=900)
    return np.load(out)


def test_debug_build_computes_what_the_release_build_computes(debug_lib, tmp_path):
    import debug_build_child as child
    from paper_1211_3991_gb300 import xyl
    dbg = _run_child(tmp_path / "debug.npz", False)
    assert str(dbg["lib"]).endswith("libxyl_debug.so")
    assert list(dbg["statuses"]) == [0] * len(child.CASES)
    assert xyl.LIB_PATH.endswith("libxyl.so")
    for k, case in enumerate(child.CASES):
        state, status = child.run_case(case)
        assert status == 0, case
        assert dbg[f"case{k}"].tobytes() == state, case


def test_debug_build_reports_an_out_of_range_neighbour_id(debug_lib, tmp_path):
    import debug_build_child as child
    from paper_1211_3991_gb300 import xyl
    bad = _run_child(tmp_path / "bad.npz", True)
    # every engine and shape met the id N + 1 and skipped it
    assert list(bad["statuses"]) == [xyl.EBOUNDS] * len(child.CASES)
