"""Parity at the limits of the C ABI: the widest grid (QV_MAX_WIDTH), the
deepest tree (QV_MAX_DEPTH), a tall narrow grid with one column of bands,
and a batch mixing those shapes."""
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


def _close(got, ref, floor=1.0, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = max(np.abs(ref).max(initial=0.0), floor)
    err = np.abs(got - ref).max(initial=0.0)
    assert err <= REL * scale, f"{what}: {err:.3e} > {REL:.0e} * {scale:.3e}"


def _run(api, w, depth, K, leaf_mode):
    m = api.Model(w)
    Qf = O.value_iteration(w)["Q"].astype(np.float32)
    Qd = m.to_grid(Qf.reshape(5, w.H, w.W))
    o = O.tree_plan(w, Qf.astype(np.float64), depth=depth, K=K)
    rep = torch.from_numpy(o["samples_flat"].copy()).cuda()
    r, plan = api.qv_tree_plan(m, Qd, m.b0(), depth=depth, K=K, seed=w.seed, episode=w.episode,
                               leaf_mode=leaf_mode, replay=rep, keep=True)
    assert r["nodes_per_level"] == [int(x) for x in o["n_level"]]
    _close(r["value"], o["root_value"], what="root value")
    _close(r["q"], o["root_q"], what="root q")
    lv = plan.level(0, depth)
    _close(lv["value"].cpu().numpy(), o["value"][depth], what="leaf values")
    assert np.array_equal(lv["obs"].cpu().numpy(), o["obs"][depth])
    return r, o


@pytest.mark.parametrize("leaf_mode", [0, 1])
def test_widest_grid(api, leaf_mode):
    from paper_1810_00204_gb300 import _native as N
    w = WL.tiny(21, H=5, W=N.QV_MAX_WIDTH)
    _run(api, w, depth=2, K=4, leaf_mode=leaf_mode)


def test_wider_than_the_limit_is_refused(api):
    from paper_1810_00204_gb300 import _native as N
    w = WL.tiny(21, H=2, W=N.QV_MAX_WIDTH + 8)
    with pytest.raises(N.QVError) as ei:
        api.Model(w)  # the model build already refuses the grid
    assert ei.value.status == N.QV_ERR_INVALID


@pytest.mark.parametrize("leaf_mode", [0, 1])
def test_deepest_tree(api, leaf_mode):
    from paper_1810_00204_gb300 import _native as N
    w = WL.tiny(22, H=6, W=7)
    w.beacons = w.beacons[:1]
    w.sense_range = 3
    _run(api, w, depth=N.QV_MAX_DEPTH, K=2, leaf_mode=leaf_mode)


def test_depth_four_mid_sized(api):
    w = WL.tiny(23, H=24, W=20)
    _run(api, w, depth=4, K=3, leaf_mode=0)


def test_tall_narrow_grid(api):
    w = WL.tiny(24, H=1500, W=3)
    _run(api, w, depth=2, K=4, leaf_mode=0)


def test_batch_of_extreme_shapes(api):
    ws = [WL.tiny(25, H=3, W=700), WL.tiny(26, H=300, W=4),
          WL.custom(1, 1, [0], [0], 1, 0, 0, 0.1, 0.9, 0.95, [1.0], depth=3, K=4),
          WL.tiny(28, H=31, W=33)]
    ms = [api.Model(w) for w in ws]
    Qs = [m.to_grid(O.value_iteration(w)["Q"].astype(np.float32).reshape(5, w.H, w.W)) for m, w in zip(ms, ws)]
    res = api.qv_tree_plan_batched(ms, Qs, [m.b0() for m in ms], depth=3, K=4, seed=9, episode=0)
    for e, w in enumerate(ws):
        Qe = ms[e].from_grid(Qs[e]).reshape(5, -1).astype(np.float64)
        o = O.tree_plan(w, Qe, depth=3, K=4, seed=9, episode=e)
        if o["boundary_count"]:
            continue
        assert res[e]["nodes_per_level"] == [int(x) for x in o["n_level"]], e
        _close(res[e]["value"], o["root_value"], what=f"episode {e}")
