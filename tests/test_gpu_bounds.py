"""GPU parity of the AEMS fields (Alg. 5-7, Eq. 9): qv_plan_bounds through
the C ABI against the oracle's tree_bounds on the oracle's own tree (the GPU
plan replays the oracle's sampled observations, so both trees are the same)
with the same leaf lower bounds, taken from the oracle; and the whole chain
on the mid map -- FIB alpha-vectors for U, PBVI for the leaves' L, bounds up
to the root -- run on the GPU and checked for the order of its bounds.

Values |d| <= 1e-5 * max(|ref|, 1).  A pointer E must equal the oracle's
unless the oracle's best and second-best gamma w H_V are within 1e-4 * scale
of each other (then the GPU's pick must be within that margin of the best)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1810_00204_gb300 import _native as N
from paper_1810_00204_gb300 import workloads as WL
from test_gpu_parity import _close

pytestmark = pytest.mark.gpu

GAP = 1e-4


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1810_00204_gb300 import api as A
    return A


def _oracle_tree_on_gpu(api, w, Qf, leaf_mode, store_levels=-1):
    """The oracle's tree on FP32-rounded alpha-vectors Qf and the GPU plan
    that replays its sampled observations (the same tree)."""
    m = api.Model(w)
    o = O.tree_plan(w, Qf.astype(np.float64), depth=w.depth, K=w.K, seed=w.seed, episode=w.episode,
                    store_levels=store_levels)
    r, plan = api.qv_tree_plan(m, m.to_grid(Qf.reshape(5, w.H, w.W)), m.b0(), depth=w.depth, K=w.K, seed=w.seed,
                               episode=w.episode, leaf_mode=leaf_mode,
                               replay=torch.from_numpy(o["samples_flat"].copy()).cuda(), keep=True)
    assert r["nodes_per_level"] == [int(x) for x in o["n_level"]]
    return m, o, r, plan


def _compare(gpu, ora, tree, gamma, scale):
    depth = tree["depth"]
    f, off = tree["flat"], tree["off"]
    for l in range(depth + 1):
        g = gpu[l]
        _close(g["LV"].cpu().numpy(), ora["LV"][l], floor=scale, what=f"L_V level {l}")
        _close(g["HV"].cpu().numpy(), ora["HV"][l], floor=scale, what=f"H_V level {l}")
        if l < depth:
            _close(g["LQ"].cpu().numpy(), ora["LQ"][l], floor=scale, what=f"L_Q level {l}")
            _close(g["HQ"].cpu().numpy(), ora["HQ"][l], floor=scale, what=f"H_Q level {l}")
            # the Q-node pointers: equal, or a near-tie of gamma w H_V
            s1, n1 = int(off[l + 1]), int(f["n_level"][l + 1])
            par, act = f["parent"][s1:s1 + n1], f["action"][s1:s1 + n1]
            h = gamma * f["weight"][s1:s1 + n1] * ora["HV"][l + 1]
            geq = g["EQ"].cpu().numpy()
            for i, a in zip(*np.nonzero(geq != ora["EQ"][l])):
                sib = np.flatnonzero((par == i) & (act == a))
                hs = h[sib]
                got = np.flatnonzero(ora["EV"][l + 1][sib] == geq[i, a])
                assert len(got) and hs[got].max() >= hs.max() - GAP * scale, f"E_Q level {l} node {i} action {a}"


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("leaf_mode", [0, 1])
def test_bounds_match_oracle_on_the_oracle_tree(api, seed, leaf_mode):
    w = WL.tiny(seed)
    Qf = O.fib_iteration(w)["alpha"].astype(np.float32)
    m, o, r, plan = _oracle_tree_on_gpu(api, w, Qf, leaf_mode)
    rng = np.random.default_rng(seed)
    U = o["value"][w.depth]
    L = (U - rng.uniform(0.0, 10.0, len(U))).astype(np.float32)
    gpu = plan.bounds(torch.from_numpy(L).cuda())
    ora = O.tree_bounds(o, L.astype(np.float64), w.discount)
    scale = max(1.0, float(np.abs(U).max()))
    _compare(gpu, ora, o, w.discount, scale)
    # the root pointer indexes the leaf level
    e = int(gpu[0]["EV"][0])
    assert 0 <= e < len(U)


def test_equal_leaf_bounds_close_the_gap(api):
    w = WL.tiny(3)
    m = api.Model(w)
    Q = api.fib_value_iterate(m)["Q"]
    r, plan = api.qv_tree_plan(m, Q, m.b0(), depth=3, K=4, seed=1, leaf_mode=1, keep=True)
    U = plan.level(0, 3)["value"]
    b = plan.bounds(U.clone())
    for l in range(4):
        lvl = plan.level(0, l)
        _close(b[l]["LV"].cpu().numpy(), lvl["value"].cpu().numpy(), floor=100.0, what=f"L_V level {l}")
        assert torch.all(b[l]["HV"] == 0)


def test_mid_fib_pbvi_chain(api):
    # the paper's node fields on the mid map, all on the GPU: U from FIB
    # leaves, L from PBVI leaves (64 points), materialised leaf beliefs; the
    # bounds keep their order
    w = WL.mid(0)
    m = api.Model(w)
    Q = api.fib_value_iterate(m)["Q"]
    g = api.pbvi_solve(m, rounds=6, iters=8, seed=2)
    r, plan = api.qv_tree_plan(m, Q, m.b0(), depth=w.depth, K=w.K, seed=w.seed, leaf_mode=N.QV_LEAF_MATERIALISE,
                               keep=True)
    leaves = plan.level(0, w.depth)
    Lleaf, _ = g["pbvi"].value(g["G"], leaves["belief"])
    U = leaves["value"]
    assert torch.all(Lleaf <= U + 1e-4 * torch.clamp(U.abs(), min=1.0))
    b = plan.bounds(Lleaf)
    scale = max(1.0, float(U.abs().max()))
    assert float(b[0]["LV"][0]) <= r["value"] + 1e-5 * scale
    assert float(b[0]["HV"][0]) >= 0.0
    for l in range(w.depth + 1):
        assert torch.all(b[l]["LV"] <= plan.level(0, l)["value"] + 1e-5 * scale)
    # against the oracle on its own mid tree (FIB alpha-vectors of the oracle),
    # the leaves' L from the oracle's pessimistic PBVI vector alpha_0
    Qf = O.fib_iteration(w)["alpha"].astype(np.float32)
    m2, o, r2, plan2 = _oracle_tree_on_gpu(api, w, Qf, N.QV_LEAF_MATERIALISE, store_levels=w.depth)
    Lo = O.pbvi_value(O.pbvi_init(w)[None, :], o["belief"][w.depth]).astype(np.float32)
    gpu = plan2.bounds(torch.from_numpy(Lo).cuda())
    ora = O.tree_bounds(o, Lo.astype(np.float64), w.discount)
    scale = max(1.0, float(np.abs(o["value"][w.depth]).max()))
    _compare(gpu, ora, o, w.discount, scale)
