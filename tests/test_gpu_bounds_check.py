"""The index-checked debug build (-DTOPO_BOUNDS_CHECK, libtopo_gb300_bc.so): the workloads of
bounds_check_cases.py run in a child process against it record no index out of range, and give
the bits of the release build (the checks only guard indices); a check that fails by construction
is recorded with its index and size, and a reset clears the record."""
import os
import subprocess
import sys

import numpy as np
import pytest

import bounds_check_cases
from gpu_helpers import topo_lib, torch_cuda

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_checked_build_records_nothing_and_gives_the_release_bits(tmp_path):
    torch = torch_cuda()
    topo = topo_lib()
    from paper_1606_06201_gb300 import build
    lib = build.build(bounds_check=True)
    out = tmp_path / "bc.npz"
    env = dict(os.environ, TOPO_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_check_cases.py"), str(out)],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    bc = np.load(out)
    assert bc["report"][0] == 0, bc["report"]
    count, index, size, after = bc["selftest"]
    assert count == 1 and index == 5 and size == 3 and after == 0
    assert not topo.bounds_check_enabled()
    rel = bounds_check_cases.run_cases(topo, torch)
    for k, v in rel.items():
        np.testing.assert_array_equal(bc[k], v, err_msg=k)
