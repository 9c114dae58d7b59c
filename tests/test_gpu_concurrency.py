"""Plans limited to part of the GPU (grid_ctas) and plans running
concurrently on several streams give the plans of the whole grid: the same
tree shapes, samples and root actions, values within FP32 summation order
(1e-5 * max(|v|, 1)), and the oracle's root value."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1810_00204_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1810_00204_gb300 import api as A
    return A


def _setup(api, n=12):
    w = WL.mid(0)
    m = api.Model(w)
    Q = m.to_grid(O.value_iteration(w)["Q"].astype(np.float32).reshape(5, w.H, w.W))  # the oracle's Q
    eps = WL.episodes(w, n, seed=3)
    return w, m, Q, eps, [m.to_grid(e.b0) for e in eps]


@pytest.mark.parametrize("grid", [1, 7, 38, 150])
def test_limited_grid_gives_the_same_plan(api, grid):
    w, m, Q, eps, b0s = _setup(api, 2)
    full = api.Plan([m], [Q], [b0s[0]], depth=w.depth, K=w.K, seed=w.seed, episode=eps[0].episode)
    part = api.Plan([m], [Q], [b0s[0]], depth=w.depth, K=w.K, seed=w.seed, episode=eps[0].episode, grid_ctas=grid)
    assert part.grid == min(grid, full.grid)
    full.run()
    part.run()
    a, b = full.read()[0], part.read()[0]
    assert a["nodes_per_level"] == b["nodes_per_level"] and a["action"] == b["action"]
    assert abs(a["value"] - b["value"]) <= 1e-5 * max(1.0, abs(a["value"]))
    assert np.allclose(a["q"], b["q"], rtol=0, atol=1e-5 * max(1.0, float(np.abs(a["q"]).max())))
    for l in range(w.depth):
        assert torch.equal(full.level(0, l)["samples"], part.level(0, l)["samples"])


def test_concurrent_streams_match_one_stream(api):
    w, m, Q, eps, b0s = _setup(api, 12)
    seq = [api.Plan([m], [Q], [b0s[i]], depth=w.depth, K=w.K, seed=w.seed, episode=e.episode)
           for i, e in enumerate(eps)]
    con = [api.Plan([m], [Q], [b0s[i]], depth=w.depth, K=w.K, seed=w.seed, episode=e.episode, grid_ctas=38)
           for i, e in enumerate(eps)]
    for p in con:
        p.capture_graph()
    streams = [torch.cuda.Stream() for _ in range(4)]
    main = torch.cuda.current_stream()
    for p in seq:
        p.run()
    for _ in range(3):  # several rounds of overlapping launches
        for s in streams:
            s.wait_stream(main)
        for i, p in enumerate(con):
            p.run(streams[i % 4])
        for s in streams:
            main.wait_stream(s)
    torch.cuda.synchronize()
    Qh = O.value_iteration(w)["Q"].astype(np.float32).astype(np.float64)  # the plans' Q
    for i, (p, q) in enumerate(zip(seq, con)):
        a, b = p.read()[0], q.read()[0]
        assert a["nodes_per_level"] == b["nodes_per_level"] and a["action"] == b["action"]
        assert abs(a["value"] - b["value"]) <= 1e-5 * max(1.0, abs(a["value"]))
        if i < 2:
            o = O.tree_plan(w, Qh, b0=eps[i].b0.ravel().astype(np.float64), episode=eps[i].episode)
            if o["boundary_count"] == 0:
                assert abs(b["value"] - o["root_value"]) <= 1e-5 * max(1.0, abs(o["root_value"]))


def test_negative_grid_is_refused(api):
    from paper_1810_00204_gb300 import _native as N
    w, m, Q, eps, b0s = _setup(api, 1)
    with pytest.raises(N.QVError) as ei:
        api.Plan([m], [Q], [b0s[0]], depth=w.depth, K=w.K, grid_ctas=-1)
    assert ei.value.status == N.QV_ERR_INVALID
