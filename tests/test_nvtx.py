"""NVTX ranges of the library's entry points, seen without a GPU: a small
NVTX tool (tests/c_client/nvtx_record.c, loaded through
NVTX_INJECTION64_PATH) records every push and pop while a child process
calls entry points whose arguments fail host-side validation.  Each call
must open its range ("qvts:<name>") and close it on the early return."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_client", "nvtx_record.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")

CHILD = r"""
import ctypes, sys
sys.path.insert(0, sys.argv[1])
from paper_1810_00204_gb300 import _native as N
L = N.lib()
assert L.qv_model_build(0, 5, 8, None, None, 1, 1, 0, None, None) == N.QV_ERR_INVALID
assert L.qv_tree_backward(None, 0, 1.0, None, None, None, None, None, None, 0, None) == N.QV_ERR_INVALID
assert L.belief_predict(None, None, 0, None, None) == N.QV_ERR_INVALID
assert L.qv_tree_plan(None, None, None, None, None, 0, None, None) == N.QV_ERR_INVALID
print("ok")
"""


def test_entry_points_open_and_close_nvtx_ranges(tmp_path):
    from paper_1810_00204_gb300 import build as B
    B.build()
    gcc = shutil.which("gcc")
    if gcc is None or not os.path.exists(os.path.join(CUDA, "include", "nvtx3", "nvToolsExt.h")):
        pytest.skip("needs gcc and the NVTX v3 headers")
    tool = str(tmp_path / "libnvtx_record.so")
    subprocess.check_call([gcc, "-std=c99", "-Wall", "-Werror", "-shared", "-fPIC", "-I",
                           os.path.join(CUDA, "include"), SRC, "-o", tool])
    log = tmp_path / "nvtx.log"
    env = dict(os.environ, NVTX_INJECTION64_PATH=tool, QVTS_NVTX_LOG=str(log))
    out = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stderr
    events = log.read_text().splitlines()
    pushed = [e[5:] for e in events if e.startswith("push ")]
    for name in ("qv_model_build", "qv_tree_backward", "belief_predict", "qv_tree_plan"):
        assert f"qvts:{name}" in pushed, (name, pushed)
    # qv_tree_plan runs through qv_tree_plan_batched: nested, both closed
    assert "qvts:qv_tree_plan_batched" in pushed
    depth = 0
    for e in events:
        depth += 1 if e.startswith("push ") else -1
        assert depth >= 0, events
    assert depth == 0, events
