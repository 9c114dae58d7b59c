"""The search's support windows: a node d levels below the root is zero
outside the bounding box of b0's nonzero cells dilated by d cells (the motion
stencil of Eq. 3 / Eq. 10 moves mass by one cell; the observation weights
only rescale), so k_plan restricts its sums to that window and writes zeros
outside it in the beliefs it stores.  Each case below compares the whole tree
with the FP64 oracle (which always sums over the whole grid): windows clipped
by the grid's edges and corners, a start belief beside the goal (the exact
stencil rows), a start belief over every free cell (no restriction), two
distant blocks (a window with a hole), and one plan object re-run with a
smaller support after a full one (the window found afresh each run, the
stored beliefs zero outside it)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1810_00204_gb300 import workloads as WL
from test_gpu_parity import _oracle_Q, compare_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1810_00204_gb300 import api as A
    return A


def _block(w, centres, half=1):
    """Uniform over the free cells of (2 half + 1)^2 blocks at `centres`."""
    b = np.zeros((w.H, w.W), np.float64)
    for (r0, c0) in centres:
        for r in range(max(0, r0 - half), min(w.H, r0 + half + 1)):
            for c in range(max(0, c0 - half), min(w.W, c0 + half + 1)):
                if not w.occ[r, c]:
                    b[r, c] = 1.0
    assert b.sum() > 0
    return (b / b.sum()).astype(np.float32)


def _with_b0(w, b):
    w.b0 = np.asarray(b, np.float32).reshape(w.H, w.W)
    return w


def _free_near(w, r, c):
    """The free cell nearest to (r, c) (Manhattan, then row-major)."""
    rr, cc = np.nonzero(w.occ == 0)
    i = np.argmin(np.abs(rr - r) + np.abs(cc - c))
    return int(rr[i]), int(cc[i])


CASES = ["corner", "edge", "goal", "everywhere", "two_blocks"]


def _case(name):
    w = WL.mid(4, H=70, W=150)
    if name == "corner":
        return _with_b0(w, _block(w, [_free_near(w, 0, w.W - 1)]))
    if name == "edge":
        return _with_b0(w, _block(w, [_free_near(w, w.H // 2, 0)], half=3))
    if name == "goal":
        g = divmod(int(w.goal), w.W)
        return _with_b0(w, _block(w, [g], half=2))
    if name == "everywhere":
        b = (1 - w.occ).astype(np.float64)
        return _with_b0(w, (b / b.sum()).astype(np.float32))
    return _with_b0(w, _block(w, [_free_near(w, 5, 10), _free_near(w, w.H - 6, w.W - 12)]))


@pytest.mark.parametrize("leaf_mode", [0, 1])
@pytest.mark.parametrize("name", CASES)
def test_window_cases_match_oracle(api, name, leaf_mode):
    w = _case(name)
    compare_tree(api, w, depth=3, K=4, leaf_mode=leaf_mode, check_beliefs=(leaf_mode == 1))


def _dilated_mask(b, d):
    r, c = np.nonzero(b)
    m = np.zeros(b.shape, bool)
    m[max(0, r.min() - d):r.max() + d + 1, max(0, c.min() - d):c.max() + d + 1] = True
    return m


def test_one_plan_rerun_with_a_smaller_support(api):
    """Run a plan from b0 over every free cell (every stored belief nonzero
    almost everywhere), then, in the same plan, from a 3x3 block: the second
    run equals a fresh plan bit for bit, and its stored beliefs are exactly
    zero outside the block's bounding box dilated by the level."""
    w = _case("everywhere")
    m = api.Model(w)
    Qd = m.to_grid(_oracle_Q(w).reshape(5, w.H, w.W))
    small = _block(w, [_free_near(w, w.H // 3, w.W // 3)])
    b0d = m.to_grid(w.b0)
    kw = dict(depth=3, K=4, seed=2, episode=0, leaf_mode=1)
    p = api.Plan([m], [Qd], [b0d], **kw)
    p.run()
    p.read()
    b0d.copy_(m.to_grid(small))
    p.run()
    got = p.read()[0]
    ref_plan = api.Plan([m], [Qd], [m.to_grid(small)], **kw)
    ref_plan.run()
    ref = ref_plan.read()[0]
    assert got["nodes_per_level"] == ref["nodes_per_level"]
    assert got["value"] == ref["value"] and got["action"] == ref["action"]
    assert np.array_equal(got["q"], ref["q"])
    for l in range(1, 4):
        a = p.level(0, l)
        b = ref_plan.level(0, l)
        assert torch.equal(a["value"], b["value"])
        ga = a["belief"].cpu().numpy()[:, :, :w.W]
        assert np.array_equal(ga, b["belief"].cpu().numpy()[:, :, :w.W])
        outside = ~_dilated_mask(small.reshape(w.H, w.W), l + 1)
        assert not ga[:, outside].any(), f"level {l}: nonzero stored belief outside the window"
    # and against the oracle
    o = O.tree_plan(w, _oracle_Q(w).astype(np.float64), depth=3, K=4, seed=2, b0=small)
    if o["boundary_count"] == 0:
        assert got["nodes_per_level"] == [int(x) for x in o["n_level"]]
        assert abs(got["value"] - o["root_value"]) <= 1e-5 * max(1.0, abs(o["root_value"]))


def test_batched_episodes_with_different_windows(api):
    """Episodes of one launch with windows of different sizes and places
    (corner, edge, everywhere) against one plan per episode."""
    ws = [_case(n) for n in ("corner", "everywhere", "edge", "two_blocks")]
    ms = [api.Model(w) for w in ws]
    Qs = [m.to_grid(_oracle_Q(w).reshape(5, w.H, w.W)) for m, w in zip(ms, ws)]
    b0s = [m.b0() for m in ms]
    batch = api.qv_tree_plan_batched(ms, Qs, b0s, depth=3, K=4, seed=3, episode=0)
    for e, m in enumerate(ms):
        one = api.qv_tree_plan(m, Qs[e], b0s[e], depth=3, K=4, seed=3, episode=e)
        assert one["nodes_per_level"] == batch[e]["nodes_per_level"]
        assert one["action"] == batch[e]["action"]
        assert one["value"] == pytest.approx(batch[e]["value"], rel=1e-5, abs=1e-5)
