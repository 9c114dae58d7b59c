"""The C ABI from plain C: tests/c_client/plan_client.c includes qvts.h as
C99, links libqvts.so and the CUDA runtime, and plans on a small grid.  The
CPU test compiles and links it (-Wall -Werror); the GPU test runs it and
checks its root result against the FP64 oracle on the same problem."""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_1810_00204_gb300 import workloads as WL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_client", "plan_client.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _build(tmp_path):
    from paper_1810_00204_gb300 import build as B
    lib = B.build()
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "plan_client")
    libdir = os.path.dirname(lib)
    subprocess.check_call([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(CUDA, "include"), SRC, "-o", exe, "-L", libdir, "-lqvts",
                           "-L", os.path.join(CUDA, "lib64"), "-lcudart", f"-Wl,-rpath,{libdir}",
                           f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}"])
    return exe


def test_c_client_compiles_and_links(tmp_path):
    assert os.path.exists(_build(tmp_path))


def _workload(H, W, seed):
    """The client's recipe, unpadded."""
    occ = np.zeros((H, W), np.uint8)
    occ[H // 2, :] = 1
    occ[H // 2, seed % W] = 0
    b0 = np.zeros((H, W), np.float32)
    b0[0:3, 1:4] = np.float32(1.0 / 9.0)
    beacons = [1 * W + 1, (H - 2) * W + (W - 2)]
    goal = (H - 1) * W + W // 2
    return WL.custom(H, W, occ, beacons, 4, goal, 1, 0.1, 0.9, 0.95, b0, depth=2, K=4, seed=seed)


@pytest.mark.gpu
@pytest.mark.parametrize("H,W,seed", [(12, 10, 3), (9, 17, 5)])
def test_c_client_matches_the_oracle(tmp_path, H, W, seed):
    exe = _build(tmp_path)
    out = subprocess.run([exe, str(H), str(W), str(seed)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    r = json.loads(out.stdout.strip().splitlines()[-1])
    w = _workload(H, W, seed)
    P = (W + 7) // 8 * 8
    assert r["goal"] == (w.goal // W) * P + w.goal % W
    vi = O.value_iteration(w, tol=1e-9)
    Qf = vi["Q"].astype(np.float32).astype(np.float64)
    o = O.tree_plan(w, Qf, depth=2, K=4, seed=seed)
    if o["boundary_count"]:
        pytest.skip("a draw fell within 1e-6 of a CDF step")
    assert r["nodes"] == [int(x) for x in o["n_level"]]
    assert abs(r["value"] - o["root_value"]) <= 1e-5 * max(1.0, abs(o["root_value"]))
    assert np.allclose(r["q"], o["root_q"], rtol=1e-5, atol=1e-5)
