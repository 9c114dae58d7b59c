"""The bounds-checked debug build (libqvts_debug.so, -DQV_BOUNDS_CHECK) on
the GPU: tests/debug_build_child.py runs the plan's parity cases against the
FP64 oracle with every device bounds check compiled in (none may fail), then
checks that an injected check failure (QVTS_FAULT=bounds) is reported as
QV_ERR_BOUNDS and that the plan recovers.  A child process, so that this
process keeps the release library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_checked_build_passes_parity_and_reports_injected_failures():
    env = dict(os.environ, QVTS_LIB="debug")
    env.pop("QVTS_FAULT", None)
    out = subprocess.run([sys.executable, os.path.join(HERE, "debug_build_child.py")], env=env,
                         capture_output=True, text=True, timeout=1200)
    tail = (out.stdout + out.stderr)[-3000:]
    assert out.returncode == 0, tail
    assert out.stdout.strip().splitlines()[-1] == "ok", tail
