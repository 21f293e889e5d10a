"""The bounds-checked build of the library (FASTCOD_CHECKED=1: every
computed index of the path's gathers, scatters and list writes is tested
and a failure is reported by the call) runs parity cases of every form in a
process of its own (tests/checked_runner.py)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def test_checked_build_matches_the_oracle():
    from paper_2302_09247_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, FASTCOD_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_runner.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "no bounds check failed" in r.stdout
