"""The autotuner of the plan kernel's launch shape (band of rows per work
item, work items per CTA): every candidate gives the oracle's tree, the
fastest is cached per shape class and picked up by later plans."""
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
    A.tune_clear()
    yield A
    A.tune_clear()


def _close(got, ref, rel=REL, floor=1.0, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = max(np.abs(ref).max(initial=0.0), floor)
    assert np.abs(got - ref).max(initial=0.0) <= rel * scale, what


def _vi(api, m):
    vi = api.mdp_value_iterate(m, dtype="f32")
    assert vi["status"] == 0
    return vi["Q"]


@pytest.mark.parametrize("band_cells,items", [(1024, 1), (2048, 2), (4096, 4), (4096, 8), (512, 3)])
def test_every_launch_shape_gives_the_oracle_tree(api, band_cells, items):
    w = WL.mid(0)
    m = api.Model(w)
    Q = _vi(api, m)  # the GPU's VI runs; the plans take the oracle's Q (in FP32)
    Qo = O.value_iteration(w)["Q"].astype(np.float32)
    Q = m.to_grid(Qo.reshape(5, w.H, w.W))
    o = O.tree_plan(w, Qo.astype(np.float64))
    rep = torch.from_numpy(o["samples_flat"].copy()).cuda()
    for leaf_mode in (0, 1):
        p = api.Plan([m], [Q], [m.b0()], depth=w.depth, K=w.K, seed=w.seed, leaf_mode=leaf_mode, replay=rep,
                     band_cells=band_cells, items_per_cta=items)
        assert p.tuning == dict(band_cells=band_cells, items_per_cta=items)
        p.run()
        r = p.read()[0]
        assert r["nodes_per_level"] == [int(x) for x in o["n_level"]]
        _close(r["value"], o["root_value"], what="root value")
        _close(r["q"], o["root_q"], what="root q")
        lv = p.level(0, w.depth)
        _close(lv["value"].cpu().numpy(), o["value"][w.depth], what="leaf values")


def test_band_too_large_for_shared_memory_is_refused(api):
    from paper_1810_00204_gb300 import _native as N
    w = WL.mid(0)
    m = api.Model(w)
    Q = _vi(api, m)
    with pytest.raises(N.QVError) as ei:
        api.Plan([m], [Q], [m.b0()], depth=3, K=8, band_cells=16384, items_per_cta=2)
    assert ei.value.status == N.QV_ERR_INVALID


def test_autotune_caches_the_fastest_shape(api):
    api.tune_clear()
    ws = WL.batched(3, E=12, lo=32, hi=96)
    ms = [api.Model(x) for x in ws]
    Qs = [_vi(api, m) for m in ms]
    b0s = [m.b0() for m in ms]
    default = api.Plan(ms, Qs, b0s, depth=3, K=8, seed=0)
    assert default.tuning == dict(band_cells=2048, items_per_cta=2)
    default.run()
    ref = default.read()
    best, table = api.autotune(ms, Qs, b0s, depth=3, K=8, seed=0, reps=3)
    assert len(table) >= 8
    assert best["ms"] == min(t["ms"] for t in table)
    tuned = api.Plan(ms, Qs, b0s, depth=3, K=8, seed=0)
    assert tuned.tuning == dict(band_cells=best["band_cells"], items_per_cta=best["items_per_cta"])
    tuned.run()
    got = tuned.read()
    for e in range(len(ws)):
        if got[e]["boundary_samples"] or ref[e]["boundary_samples"]:
            continue
        assert got[e]["nodes_per_level"] == ref[e]["nodes_per_level"]
        _close(got[e]["value"], ref[e]["value"], what=f"episode {e}")
    # another shape class keeps the defaults
    other = api.Plan(ms[:1], Qs[:1], b0s[:1], depth=2, K=4, seed=0)
    assert other.tuning == dict(band_cells=2048, items_per_cta=2)
    api.tune_clear()
    again = api.Plan(ms, Qs, b0s, depth=3, K=8, seed=0)
    assert again.tuning == dict(band_cells=2048, items_per_cta=2)
