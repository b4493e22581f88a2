"""The checked build (libhalftime_check.so: every global access of the
warp-chunk kernels range-checked, out-of-range accesses recorded and
skipped) runs single strings, batches (aligned and not), both block sizes,
incremental pieces and split parts without a single check firing, and with
digests equal to the oracle's.  It stands in for a memory checker, which is
not available on every GPU host.  Runs in a child process, since the
library is chosen when the binding is imported."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_runs_clean(built):
    env = dict(os.environ, HALFTIME_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "checked: ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
