"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (FP32 kernels against FP64): beliefs |d| <= 1e-5 * max|ref|
elementwise; values, rewards and Q-values |d| <= 1e-5 * max(|ref|, 1);
sampled observations identical except where the oracle flags the uniform as
lying within 1e-6 of a CDF step (then the oracle's samples are replayed);
chosen actions identical unless the two best Q-values are within 1e-5.
"""
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


def _rand_belief(w, seed):
    rng = np.random.default_rng(seed)
    b = rng.random(w.H * w.W) * (1 - w.occ.ravel())
    return (b / b.sum()).astype(np.float32)


def _close(got, ref, rel=REL, floor=0.0, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = max(np.abs(ref).max(initial=0.0), floor)
    err = np.abs(got - ref).max(initial=0.0)
    assert err <= rel * scale + 1e-30, f"{what}: max err {err:.3e} > {rel:.0e} * {scale:.3e}"


WORKLOADS = [
    lambda: WL.tiny(0),
    lambda: WL.tiny(5, H=13, W=17),        # ragged width (pitch 20) and height
    lambda: WL.mid(1, H=67, W=45),
    lambda: WL.batched(2, E=1, lo=40, hi=90)[0],
]


# ------------------------------------------------------------------ model build
@pytest.mark.parametrize("make", WORKLOADS)
def test_model_build_labels_and_free(api, make):
    w = make()
    m = api.Model(w)
    cell = m.cell.cpu().numpy().view(np.uint16)[:, :w.W].reshape(-1).astype(np.int64)
    assert np.array_equal((cell >> 8) & 0x7F, O.labels(w))
    assert np.array_equal(cell >> 15, 1 - w.occ.reshape(-1))


# ------------------------------------------------------------------ predict / correct / leaf
@pytest.mark.parametrize("make", WORKLOADS)
def test_belief_predict_parity(api, make):
    w = make()
    m = api.Model(w)
    for s in range(2):
        b = _rand_belief(w, s)
        bd = m.to_grid(b.reshape(w.H, w.W))
        for a in range(5):
            got = m.from_grid(api.belief_predict(m, bd, a))
            ref = O.predict(w, b.astype(np.float64), a)
            _close(got, ref, what=f"predict a={a}")
            assert got.sum() == pytest.approx(ref.sum(), rel=1e-5)


@pytest.mark.parametrize("make", WORKLOADS)
def test_belief_correct_parity(api, make):
    w = make()
    m = api.Model(w)
    lab = O.labels(w)
    b = _rand_belief(w, 3)
    for a in (0, 2, 4):
        bbar = O.predict(w, b.astype(np.float64), a).astype(np.float32)
        bd = m.to_grid(bbar.reshape(w.H, w.W))
        for z in range(w.B + 1):
            got, pz = api.belief_correct(m, bd, z)
            ref, rpz = O.correct(w, bbar.astype(np.float64), z, lab)
            _close(m.from_grid(got), ref, what=f"correct z={z}")
            assert float(pz.item()) == pytest.approx(rpz, rel=1e-5)


def test_leaf_value_parity(api):
    w = WL.mid(2, H=40, W=36)
    m = api.Model(w)
    vi = O.value_iteration(w)
    Qf = vi["Q"].astype(np.float32)
    Qd = m.to_grid(Qf.reshape(5, w.H, w.W))
    bs = np.stack([_rand_belief(w, s) for s in range(6)])
    got = api.leaf_value(m, Qd, m.to_grid(bs.reshape(6, w.H, w.W))).cpu().numpy()
    ref = [O.leaf_value(w, Qf.astype(np.float64), b.astype(np.float64))[0] for b in bs]
    _close(got, ref, floor=1.0, what="leaf")


# ------------------------------------------------------------------ value iteration
def test_vi_f64_tiny(api):
    for s in range(3):
        w = WL.tiny(s)
        m = api.Model(w)
        r = api.mdp_value_iterate(m, dtype="f64", tol=1e-6)
        assert r["status"] == 0 and r["residual"] < 1e-6
        o = O.value_iteration(w, truncated=r["sweeps"])
        own = O.value_iteration(w, tol=1e-6)
        assert abs(own["sweeps"] - r["sweeps"]) <= 1
        _close(m.from_grid(r["V"]), o["V"], rel=1e-12, floor=1.0, what="V f64")
        _close(m.from_grid(r["Q"]), o["Q"], rel=1e-6, floor=1.0, what="Q f64->f32")


@pytest.mark.parametrize("make", [lambda: WL.mid(0), lambda: WL.tiny(2, H=31, W=29),
                                  lambda: WL.batched(4, E=1, lo=60, hi=200)[0]])
def test_vi_f32_sweep_for_sweep(api, make):
    w = make()
    m = api.Model(w)
    r = api.mdp_value_iterate(m, dtype="f32", tol=1e-5)
    assert r["status"] == 0 and r["residual"] < 1e-5
    o = O.value_iteration(w, truncated=r["sweeps"])
    _close(m.from_grid(r["V"]), o["V"], floor=1.0, what="V f32")
    _close(m.from_grid(r["Q"]), o["Q"], floor=1.0, what="Q f32")


def test_vi_truncated_with_cost_map(api):
    w = WL.diff(0, H=48, W=40)
    m = api.Model(w)
    r = api.mdp_value_iterate(m, dtype="f32", truncated=200)
    assert r["sweeps"] == 200
    o = O.value_iteration(w, truncated=200)
    _close(m.from_grid(r["V"]), o["V"], floor=1.0, what="V cost")
    _close(m.from_grid(r["Q"]), o["Q"], floor=1.0, what="Q cost")


def test_vi_not_converged_is_reported(api):
    w = WL.tiny(1)
    m = api.Model(w)
    r = api.mdp_value_iterate(m, dtype="f32", tol=1e-5, max_sweeps=5)
    assert r["status"] == 5 and r["sweeps"] == 5


# ------------------------------------------------------------------ tree
def _oracle_Q(w):
    vi = O.value_iteration(w)
    return vi["Q"].astype(np.float32)


def compare_tree(api, w, depth, K, leaf_mode, weight_mode=0, seed=None, check_beliefs=True, Qf=None,
                 deepest_form=0):
    """Run both sides on the same inputs (leaf alpha-vectors Qf, float32
    [5][n], the oracle's QMDP ones by default); return (gpu result, oracle tree).
    deepest_form: the GPU's form of the deepest fused level (QV_DEEPEST_*)."""
    seed = w.seed if seed is None else seed
    m = api.Model(w)
    Qf = _oracle_Q(w) if Qf is None else Qf
    Qd = m.to_grid(Qf.reshape(5, w.H, w.W))
    b0 = m.b0()
    o = O.tree_plan(w, Qf.astype(np.float64), depth=depth, K=K, seed=seed, weight_mode=weight_mode,
                    store_levels=depth if check_beliefs else -1)
    replay = None
    r, plan = api.qv_tree_plan(m, Qd, b0, depth=depth, K=K, seed=seed, episode=w.episode,
                               weight_mode=weight_mode, leaf_mode=leaf_mode, keep=True, deepest_form=deepest_form)
    # sampled observations: identical except at flagged CDF boundaries
    for l in range(depth):
        lv = plan.level(0, l)
        n = lv["count"]
        if n != o["n_level"][l]:
            break
        gs = lv["samples"].cpu().numpy()
        os_ = o["samples"][l]
        bad = (gs != os_) & (o["boundary"][l] == 0)
        assert not bad.any(), f"level {l}: {int(bad.sum())} samples differ away from a CDF boundary"
        if (gs != os_).any():
            replay = torch.from_numpy(o["samples_flat"].copy()).cuda()
    if replay is not None or list(r["nodes_per_level"]) != [int(x) for x in o["n_level"]]:
        assert o["boundary_count"] > 0, "tree shapes differ without a boundary sample"
        r, plan = api.qv_tree_plan(m, Qd, b0, depth=depth, K=K, seed=seed, episode=w.episode,
                                   weight_mode=weight_mode, leaf_mode=leaf_mode,
                                   replay=torch.from_numpy(o["samples_flat"].copy()).cuda(), keep=True,
                                   deepest_form=deepest_form)
    assert r["nodes_per_level"] == [int(x) for x in o["n_level"]]
    for l in range(depth + 1):
        lv = plan.level(0, l)
        if l > 0:
            assert np.array_equal(lv["parent"].cpu().numpy(), o["parent"][l])
            assert np.array_equal(lv["action"].cpu().numpy(), o["action"][l])
            assert np.array_equal(lv["obs"].cpu().numpy(), o["obs"][l])
            _close(lv["weight"].cpu().numpy(), o["weight"][l], rel=1e-6, floor=1.0, what=f"weight l{l}")
            _close(lv["pz"].cpu().numpy(), o["pz"][l], rel=REL, floor=1e-30, what=f"pz l{l}")
        if l < depth:
            _close(lv["R"].cpu().numpy(), o["R"][l], floor=1.0, what=f"R l{l}")
            _close(lv["UQ"].cpu().numpy(), o["UQ"][l], floor=1.0, what=f"UQ l{l}")
        _close(lv["value"].cpu().numpy(), o["value"][l], floor=1.0, what=f"value l{l}")
        if check_beliefs and 0 < l and lv["belief"] is not None:
            gb = m.from_grid(lv["belief"])
            for j in range(gb.shape[0]):
                _close(gb[j], o["belief"][l][j], what=f"belief l{l} node {j}")
    _close(r["value"], o["root_value"], floor=1.0, what="root value")
    _close(r["q"], o["root_q"], floor=1.0, what="root q")
    q = np.sort(o["root_q"])
    if q[-1] - q[-2] > REL * max(1.0, abs(q[-1])):
        assert r["action"] == o["root_action"]
    return r, o


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("leaf_mode", [0, 1])
def test_tree_tiny(api, seed, leaf_mode):
    w = WL.tiny(seed)
    compare_tree(api, w, depth=2, K=4, leaf_mode=leaf_mode)


@pytest.mark.parametrize("make,depth,K", [(lambda: WL.tiny(1), 2, 4), (lambda: WL.tiny(2, H=17, W=23), 3, 5),
                                          (lambda: WL.mid(0), 3, 8)])
def test_deepest_level_in_both_forms(api, make, depth, K):
    """The deepest fused level in its per-child stencil form (QV_DEEPEST_STENCIL,
    also the form a plan falls back to when the contraction's records do not
    fit) and in its contraction form (the default), each against the oracle
    tree, and the two roots against each other within the value tolerance."""
    from paper_1810_00204_gb300 import _native as N
    w = make()
    rs, o = compare_tree(api, w, depth, K, 0, deepest_form=N.QV_DEEPEST_STENCIL, check_beliefs=False)
    rc, _ = compare_tree(api, w, depth, K, 0, deepest_form=N.QV_DEEPEST_AUTO, check_beliefs=False)
    _close(np.array([rc["value"]]), np.array([rs["value"]], np.float64), floor=1.0, what="root value, two forms")
    _close(rc["q"], rs["q"].astype(np.float64), floor=1.0, what="root q, two forms")


@pytest.mark.parametrize("weight_mode", [0, 1])
def test_tree_weight_modes(api, weight_mode):
    w = WL.tiny(7, H=15, W=22)
    compare_tree(api, w, depth=3, K=6, leaf_mode=0, weight_mode=weight_mode)


@pytest.mark.parametrize("leaf_mode", [0, 1])
def test_tree_mid_full_config(api, leaf_mode):
    """The 128x128, depth-3, K=8 configuration the benchmark times."""
    w = WL.mid(0)
    compare_tree(api, w, depth=3, K=8, leaf_mode=leaf_mode, check_beliefs=(leaf_mode == 1))


@pytest.mark.parametrize("seed", [1, 2])
def test_tree_mid_other_seeds(api, seed):
    w = WL.mid(seed)
    compare_tree(api, w, depth=3, K=8, leaf_mode=0, check_beliefs=False)


def test_tree_ragged_sizes(api):
    for (H, W) in ((5, 3), (1, 9), (9, 1), (37, 131)):
        w = WL.tiny(11, H=H, W=W)
        compare_tree(api, w, depth=2, K=5, leaf_mode=1)


def test_tree_depth0_is_qmdp(api):
    w = WL.tiny(3)
    r, o = compare_tree(api, w, depth=0, K=4, leaf_mode=0)
    assert r["nodes_per_level"] == [1]


def test_tree_edge_parameters(api):
    base = WL.tiny(6, H=12, W=14)
    for slip, acc, K in ((0.0, 0.9, 1), (0.5, 0.9, 4), (0.1, 1.0, 8), (0.1, 0.2, 64)):
        w = WL.tiny(6, H=12, W=14)
        w.slip, w.accuracy = slip, acc
        compare_tree(api, w, depth=2, K=K, leaf_mode=0)
    assert base.B == 4


def test_tree_single_cell_goal(api):
    w = WL.custom(1, 1, [0], [0], 1, 0, 0, 0.1, 0.9, 0.95, [1.0], depth=2, K=3)
    r, o = compare_tree(api, w, depth=2, K=3, leaf_mode=1)
    assert r["value"] == 0.0


def test_tree_many_beacons(api):
    w = WL.mid(3, H=40, W=60)
    rng = np.random.default_rng(0)
    free = np.flatnonzero(w.occ.ravel() == 0)
    w.beacons = np.sort(rng.choice(free, size=126, replace=False)).astype(np.int32)
    w.sense_range = 2
    compare_tree(api, w, depth=2, K=8, leaf_mode=0)


def test_graph_capture_matches_eager(api):
    w = WL.mid(0)
    m = api.Model(w)
    Qd = m.to_grid(_oracle_Q(w).reshape(5, w.H, w.W))
    p = api.Plan([m], [Qd], [m.b0()], depth=3, K=8, seed=0)
    p.run()
    eager = p.read()[0]
    p.capture_graph()
    for _ in range(3):
        p.run()
        g = p.read()[0]
        assert g["nodes_per_level"] == eager["nodes_per_level"]
        assert g["action"] == eager["action"]
        assert g["value"] == pytest.approx(eager["value"], rel=1e-6)


def test_batched_matches_plain(api):
    ws = WL.batched(5, E=6, lo=24, hi=70)
    ms = [api.Model(w) for w in ws]
    Qs = [m.to_grid(_oracle_Q(w).reshape(5, w.H, w.W)) for m, w in zip(ms, ws)]
    b0s = [m.b0() for m in ms]
    batch = api.qv_tree_plan_batched(ms, Qs, b0s, depth=3, K=8, seed=5, episode=0)
    for e, (w, m) in enumerate(zip(ws, ms)):
        one = api.qv_tree_plan(m, Qs[e], b0s[e], depth=3, K=8, seed=5, episode=e)
        assert one["nodes_per_level"] == batch[e]["nodes_per_level"]
        assert one["action"] == batch[e]["action"]
        assert one["value"] == pytest.approx(batch[e]["value"], rel=1e-5, abs=1e-5)
        o = O.tree_plan(w, _oracle_Q(w).astype(np.float64), depth=3, K=8, seed=5, episode=e)
        if o["boundary_count"] == 0:
            assert batch[e]["nodes_per_level"] == [int(x) for x in o["n_level"]]
            assert abs(batch[e]["value"] - o["root_value"]) <= REL * max(1.0, abs(o["root_value"]))
        else:
            # a draw at a CDF step: the oracle's samples replayed give its tree
            rp = api.qv_tree_plan(m, Qs[e], b0s[e], depth=3, K=8, seed=5, episode=e,
                                  replay=torch.from_numpy(o["samples_flat"].copy()).cuda())
            assert rp["nodes_per_level"] == [int(x) for x in o["n_level"]]
            assert abs(rp["value"] - o["root_value"]) <= REL * max(1.0, abs(o["root_value"]))


def test_async_readback_matches_read(api):
    w = WL.mid(0)
    m = api.Model(w)
    Qd = m.to_grid(_oracle_Q(w).reshape(5, w.H, w.W))
    plans = [api.Plan([m], [Qd], [m.b0()], depth=3, K=8, seed=0, episode=e) for e in range(3)]
    bufs = [p.readback_buffer() for p in plans]
    for p, b in zip(plans, bufs):
        p.run()
        p.read_async(b)
    torch.cuda.current_stream().synchronize()
    got = [p.decode(b)[0] for p, b in zip(plans, bufs)]
    ref = [p.read()[0] for p in plans]
    for g, r in zip(got, ref):
        assert g["nodes_per_level"] == r["nodes_per_level"]
        assert g["value"] == r["value"] and g["action"] == r["action"]
        assert np.array_equal(g["q"], r["q"])
