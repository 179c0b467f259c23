"""The checked build (-DWC_CHECKED, build.py --checked): index checks on
every computed site, neighbour, block-local and shared-memory index of the
operator, even-odd, RAS and multi-RHS kernels, and NaN-poisoned RAS shared
memory.  The small odd-extent parity cases of checked_cases.py run against
it in a fresh process; they must agree with the oracle and count no
out-of-range index.  (This stands in for a memory checker, which is not
available here.)"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_parity_without_out_of_range_indices():
    sys.path.insert(0, ROOT)
    import __graft_entry__
    lib = __graft_entry__._load_builder().build(checked=True)
    env = dict(os.environ, WC_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "out-of-range indices: 0" in r.stdout
