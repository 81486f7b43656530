"""The checked build (VRNERF_CHECKED=1: device-side bounds checks that record
a bit and skip the access) runs every entry point family without a failed
check, and reports a check that fires."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_runs_clean():
    env = dict(os.environ, VRNERF_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_workload.py")], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked workload OK" in r.stdout
