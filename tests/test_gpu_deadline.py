"""The anytime stop of QV-Tree Search (Sec. IV-C; Alg. 1 plans while time
permits): qv_plan_params_t.deadline_ms.  A budget that has run out by the
time the root level is final gives the depth-1 plan (the root's children
are the leaves, valued by Eq. 4), which must be the oracle's depth-1 plan;
a budget that never runs out gives the full plan, the oracle's full-depth
plan and the plan without a deadline.  Tolerances as in the other parity
tests (values |d| <= 1e-5 max(|ref|, 1), tree shape and actions exact)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1810_00204_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1810_00204_gb300 import api as A
    return A


def _case(api, w):
    m = api.Model(w)
    Qf = O.value_iteration(w)["Q"].astype(np.float32)
    return m, Qf, m.to_grid(Qf.reshape(5, w.H, w.W))


def _check(r, o, what):
    assert r["nodes_per_level"][:len(o["n_level"])] == [int(x) for x in o["n_level"]], what
    assert abs(r["value"] - o["root_value"]) <= REL * max(1.0, abs(o["root_value"])), what
    assert np.abs(np.asarray(r["q"], np.float64) - o["root_q"]).max() <= REL * max(1.0, np.abs(o["root_q"]).max())
    q = np.sort(o["root_q"])
    if q[-1] - q[-2] > REL * max(1.0, abs(q[-1])):
        assert r["action"] == o["root_action"], what


@pytest.mark.parametrize("make", [lambda: WL.mid(0), lambda: WL.tiny(3, H=23, W=31), lambda: WL.large(0)])
def test_expired_deadline_gives_the_depth_one_plan(api, make):
    w = make()
    m, Qf, Qd = _case(api, w)
    r, plan = api.qv_tree_plan(m, Qd, m.b0(), depth=w.depth, K=w.K, seed=w.seed, deadline_ms=1e-6, keep=True)
    assert r["depth_reached"] == 1
    assert all(n == 0 for n in r["nodes_per_level"][2:])
    o = O.tree_plan(w, Qf.astype(np.float64), depth=1, K=w.K, seed=w.seed)
    assert o["boundary_count"] == 0
    _check(r, o, "depth-1")
    # the leaves' records are those of the oracle's depth-1 tree
    lv = plan.level(0, 1)
    assert np.array_equal(lv["obs"].cpu().numpy(), o["obs"][1])
    assert np.array_equal(lv["action"].cpu().numpy(), o["action"][1])
    v = lv["value"].cpu().numpy()
    assert np.abs(v - o["value"][1]).max() <= REL * max(1.0, np.abs(o["value"][1]).max())


@pytest.mark.parametrize("make", [lambda: WL.mid(0), lambda: WL.tiny(3, H=23, W=31)])
def test_generous_deadline_gives_the_full_plan(api, make):
    w = make()
    m, Qf, Qd = _case(api, w)
    r = api.qv_tree_plan(m, Qd, m.b0(), depth=w.depth, K=w.K, seed=w.seed, deadline_ms=1e6)
    plain = api.qv_tree_plan(m, Qd, m.b0(), depth=w.depth, K=w.K, seed=w.seed)
    assert r["depth_reached"] == w.depth == plain["depth_reached"]
    assert r["nodes_per_level"] == plain["nodes_per_level"]
    assert r["action"] == plain["action"]
    assert abs(r["value"] - plain["value"]) <= REL * max(1.0, abs(plain["value"]))
    o = O.tree_plan(w, Qf.astype(np.float64), depth=w.depth, K=w.K, seed=w.seed)
    if o["boundary_count"] == 0:
        _check(r, o, "full depth")


def test_deadline_repeats_and_clears(api):
    # a run cut short leaves no deeper level behind for the next run
    w = WL.mid(1)
    m, Qf, Qd = _case(api, w)
    p_cut = api.Plan([m], [Qd], [m.b0()], depth=3, K=8, seed=w.seed, deadline_ms=1e-6)
    for _ in range(3):
        p_cut.run()
        r = p_cut.read()[0]
        assert r["depth_reached"] == 1 and r["nodes_per_level"][2:] == [0, 0]
    p_cut.capture_graph()
    p_cut.run()
    assert p_cut.read()[0]["depth_reached"] == 1


def test_deadline_arguments(api):
    from paper_1810_00204_gb300 import _native as N
    w = WL.tiny(0)
    m, Qf, Qd = _case(api, w)
    with pytest.raises(N.QVError) as ei:
        api.qv_tree_plan(m, Qd, m.b0(), depth=2, K=4, deadline_ms=-1.0)
    assert ei.value.status == N.QV_ERR_INVALID
    with pytest.raises(N.QVError) as ei:
        api.qv_tree_plan(m, Qd, m.b0(), depth=2, K=4, deadline_ms=1.0, leaf_mode=N.QV_LEAF_MATERIALISE)
    assert ei.value.status == N.QV_ERR_INVALID
