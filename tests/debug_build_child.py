"""Child process of tests/test_gpu_debug_build.py, started with
QVTS_LIB=debug: the package then loads the bounds-checked debug build
(libqvts_debug.so), whose plan kernel checks its workspace indices, band
copies and stored-belief offsets and reports QV_ERR_BOUNDS instead of
faulting.

1. Parity cases of the plan (tests/test_gpu_parity.py, test_gpu_windows.py,
   test_gpu_deadline.py) run against the FP64 oracle on this build: every
   check must pass (a failure raises QVError with QV_ERR_BOUNDS).
2. QVTS_FAULT=bounds makes the node-record check report a failure with its
   index in range (its write still runs): the read must raise QV_ERR_BOUNDS
   naming the site, and the next run without the variable must give the
   oracle's result again.
Prints "ok" at the end."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path[:0] = [ROOT, HERE]
assert os.environ.get("QVTS_LIB") == "debug", "run with QVTS_LIB=debug"

import numpy as np  # noqa: E402

from paper_1810_00204_gb300 import build as B  # noqa: E402

B.build(debug=True)

import oracle as O  # noqa: E402
from paper_1810_00204_gb300 import _native as N  # noqa: E402
from paper_1810_00204_gb300 import api  # noqa: E402
from paper_1810_00204_gb300 import workloads as WL  # noqa: E402

import test_gpu_deadline as TD  # noqa: E402
import test_gpu_parity as TP  # noqa: E402
import test_gpu_windows as TW  # noqa: E402

assert N.LIB_PATH.endswith("libqvts_debug.so"), N.LIB_PATH

# 1. parity with every bounds check compiled in
for seed in (0, 1):
    for leaf_mode in (0, 1):
        TP.test_tree_tiny(api, seed, leaf_mode)
for leaf_mode in (0, 1):
    TP.test_tree_mid_full_config(api, leaf_mode)
TP.test_tree_ragged_sizes(api)
TP.test_tree_many_beacons(api)
TP.test_tree_depth0_is_qmdp(api)
TP.test_batched_matches_plain(api)
for name in TW.CASES:
    TW.test_window_cases_match_oracle(api, name, 0)
TW.test_batched_episodes_with_different_windows(api)
TD.test_expired_deadline_gives_the_depth_one_plan(api, lambda: WL.mid(0))
print("parity cases passed on the bounds-checked build", flush=True)

# 2. an injected check failure is reported, and the plan recovers
w = WL.mid(0)
m = api.Model(w)
Qf = TP._oracle_Q(w)
Qd = m.to_grid(Qf.reshape(5, w.H, w.W))
o = O.tree_plan(w, Qf.astype(np.float64))
assert o["boundary_count"] == 0
p = api.Plan([m], [Qd], [m.b0()], depth=w.depth, K=w.K, seed=w.seed, episode=w.episode)
os.environ["QVTS_FAULT"] = "bounds"
p.run()
try:
    p.read()
except N.QVError as ex:
    assert ex.status == N.QV_ERR_BOUNDS, ex
    assert "node record" in str(ex), ex
else:
    raise AssertionError("the injected bounds failure was not reported")
del os.environ["QVTS_FAULT"]
for _ in range(2):
    p.run()
    r = p.read()[0]
    assert r["nodes_per_level"] == [int(x) for x in o["n_level"]]
    assert abs(r["value"] - o["root_value"]) <= 1e-5 * max(1.0, abs(o["root_value"]))
    q = np.sort(o["root_q"])
    if q[-1] - q[-2] > 1e-5 * max(1.0, abs(q[-1])):
        assert r["action"] == o["root_action"]
print("ok", flush=True)
