"""The bounds-checked debug build (libghostmg_checked.so, -DMG_CHECK_BOUNDS)
on the GPU.

Its kernels check every node index, boundary-row index and boundary-list
position where it is formed; a failed check would set a device word (and
every synchronizing call would return MG_ERR_INTERNAL) instead of faulting.
tests/bounds_workload.py runs every GPU path of the library on small and
medium problems (fp64 and mixed V-cycles with and without fused steps and
band sweeps, W-cycle, two-grid, re-discretised coarse operators, the global
constant, Neumann and box-side conditions, the adjoint and the transposed
cycle, the allocation-free residual, the batched solver, the 1D model) in a
child process per build: with the checked build no check fails and every
call returns MG_OK, and the results equal those of the normal build (the
checks change no arithmetic).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_child(checked: bool):
    env = dict(os.environ)
    env.pop("GHOSTMG_CHECKED", None)
    if checked:
        env["GHOSTMG_CHECKED"] = "1"
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_workload.py")],
                       env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.fixture(scope="module")
def results():
    from paper_2505_05105_gb300 import build
    build.build(checked=True)
    return run_child(True), run_child(False)


def test_checked_build_stays_in_bounds(results):
    checked, normal = results
    assert checked["checked"] and not normal["checked"]
    assert checked["hits"] == 0 and normal["hits"] == 0
    bad = {k: v["status"] for k, v in checked["runs"].items() if v["status"] != 0}
    assert not bad, bad


def test_checked_build_gives_the_normal_results(results):
    checked, normal = results
    assert set(checked["runs"]) == set(normal["runs"])
    for name, rc in checked["runs"].items():
        rn = normal["runs"][name]
        assert rn["status"] == 0, (name, rn["status"])
        np.testing.assert_allclose(rc["sum"], rn["sum"], rtol=1e-12, atol=0, err_msg=name)
