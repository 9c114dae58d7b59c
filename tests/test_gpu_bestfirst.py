"""GPU parity of the best-first planning loop (Alg. 1 with Alg. 2-7, Eq. 9):
the qv_bf_* calls against the oracle's bestfirst on the same upper-bound
alpha-vectors and PBVI vectors.  The oracle runs its own loop.  At the
iterations where it reports a near-tie among the comparisons that chose its
node (margin within 1e-5 * scale: FP32 and FP64 may order those
differently) the oracle's choice is replayed into the GPU loop
(qv_bf_set_replay); at every other iteration the GPU chooses on its own and
must expand the oracle's node.  Then the same tree (parents, actions,
observations, depths, weights exactly), beliefs |d| <= 1e-5 max|ref|,
fields |d| <= 1e-5 max(|ref|, 1); the stop rules; and on the full mid map
the same loop for 30 iterations."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1810_00204_gb300 import workloads as WL
from test_gpu_parity import _close

pytestmark = pytest.mark.gpu

TIE = 1e-5


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1810_00204_gb300 import api as A
    return A


def _inputs(api, w, rounds=3, iters=8):
    m = api.Model(w)
    Qu = O.fib_iteration(w)["alpha"].astype(np.float32)
    G = O.pbvi_solve(w, rounds=rounds, iters=iters)["G"].astype(np.float32)
    pb = api.Pbvi(m, max(8, G.shape[0]))
    pb.set_points(m.b0()[None])
    return m, Qu, G, pb


def _run_both(api, w, iters, K, max_depth, max_nodes=None):
    m, Qu, G, pb = _inputs(api, w)
    Qd = m.to_grid(Qu.reshape(5, w.H, w.W))
    Gd = m.to_grid(G.reshape(-1, w.H, w.W))
    nz = w.B + 1
    mn = max_nodes or 1 + iters * 5 * min(K, nz)
    o = O.bestfirst(w, Qu.astype(np.float64), G.astype(np.float64), iters, K=K, max_depth=max_depth, max_nodes=mn)
    scale = max(1.0, float(np.abs(o["U"]).max()), float(np.abs(o["L"]).max()))
    it = o["iterations"]
    near = np.zeros(iters, bool)
    near[:it] = o["margin"][:it] <= TIE * scale
    replay = np.where(near, o["expanded"], -1).astype(np.int32)
    bf = api.BestFirst(m, Qd, pb, Gd, K=K, seed=w.seed, episode=w.episode, max_depth=max_depth, max_nodes=mn)
    bf.set_replay(replay)
    bf.reset()
    bf.run(iters)
    r = bf.read()
    t = bf.tree()
    return m, bf, r, t, o


def _compare(m, r, t, o):
    assert o["boundary"] == 0 and r["boundary_samples"] == 0
    assert r["iterations"] == o["iterations"]
    assert r["nodes"] == o["nodes"]
    it = o["iterations"]
    # the GPU's own choices (every iteration not replayed) are the oracle's
    assert np.array_equal(t["expanded"][:it], o["expanded"][:it])
    for k in ("parent", "action", "obs", "depth"):
        assert np.array_equal(t[k], o[k]), k
    assert np.array_equal(t["weight"], o["weight"].astype(np.float32))
    assert np.array_equal(t["E"], o["E"])
    scale = max(1.0, float(np.abs(o["U"]).max()), float(np.abs(o["L"]).max()))
    for k in ("U", "L", "H"):
        _close(t[k], o[k], floor=scale, what=k)
    for k in ("R", "UQ", "LQ", "HQ"):
        _close(t[k], o[k], floor=scale, what=k)
    assert np.array_equal(t["first"], o["first"]) and np.array_equal(t["count"], o["count"])
    gb = m.from_grid(t["belief"]).reshape(r["nodes"], -1)
    for c in range(r["nodes"]):
        _close(gb[c], o["belief"][c], what=f"belief {c}")
    assert r["root_action"] == o["root_action"]
    _close(r["U"], o["U"][0], floor=scale, what="root U")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bestfirst_matches_oracle(api, seed):
    w = WL.tiny(seed, H=12, W=13)
    m, bf, r, t, o = _run_both(api, w, 20, K=4, max_depth=5)
    _compare(m, r, t, o)


def test_bestfirst_stops_at_the_depth_limit(api):
    w = WL.tiny(4, H=10, W=11)
    m, bf, r, t, o = _run_both(api, w, 60, K=3, max_depth=2)
    assert o["iterations"] < 60 and r["stopped"] == 1
    _compare(m, r, t, o)
    assert np.all(t["H"][t["depth"] >= 2] == 0.0)


def test_bestfirst_stops_at_capacity(api):
    w = WL.tiny(5, H=10, W=11)
    m, bf, r, t, o = _run_both(api, w, 30, K=4, max_depth=6, max_nodes=60)
    assert r["stopped"] == 1 and r["nodes"] <= 60
    _compare(m, r, t, o)
    # later calls do nothing once stopped
    bf.run(5)
    assert bf.read()["iterations"] == r["iterations"]


def test_bestfirst_mid_map(api):
    # the full mid map: FIB upper bound, an 8-point PBVI lower bound
    w = WL.mid(0)
    m, bf, r, t, o = _run_both(api, w, 30, K=8, max_depth=6)
    _compare(m, r, t, o)
    assert np.all(t["L"] <= t["U"] + 1e-4 * np.maximum(1.0, np.abs(t["U"])))
