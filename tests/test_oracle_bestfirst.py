"""Pins for the oracle's best-first QV-Tree Search (Alg. 1's planning loop
with Alg. 2-7 and Eq. 9): every node it creates is the node of the same
path in the level-synchronous tree (same samples, belief, weight and leaf
value); one expansion of the root is the depth-1 level-synchronous tree with
its AEMS fields; each iteration expands the root's E of the tree before it;
the root's E is reached by the greedy actions and the largest gamma w H_V
children, with the root's H the product along that path; lower bounds stay
below upper bounds; nodes at the depth limit are closed; each iteration's
margin is the smallest gap of the comparisons on the pointer path.  None of
these call the CUDA library."""
import numpy as np
import pytest

import oracle as O
from paper_1810_00204_gb300 import workloads as WL


def _setup(seed, H=12, W=13, K=4):
    w = WL.tiny(seed, H=H, W=W, depth=3, K=K)
    Qu = O.fib_iteration(w)["alpha"]
    G = O.pbvi_solve(w, rounds=3, iters=8)["G"]
    return w, Qu, G


@pytest.mark.parametrize("seed", [0, 1])
def test_nodes_are_the_level_synchronous_trees_nodes(seed):
    w, Qu, G = _setup(seed)
    r = O.bestfirst(w, Qu, G, 25, max_depth=4)
    D = int(r["depth"].max())
    t = O.tree_plan(w, Qu, depth=D, K=w.K, store_levels=D)
    # index the full-width tree by path: (parent index, action, z) per level
    key = [dict()] + [{(int(t["parent"][l][j]), int(t["action"][l][j]), int(t["obs"][l][j])): j
                       for j in range(int(t["n_level"][l]))} for l in range(1, D + 1)]
    where = np.zeros(r["nodes"], np.int64)   # best-first node -> index in its level
    for c in range(1, r["nodes"]):
        l = int(r["depth"][c])
        j = key[l][(int(where[r["parent"][c]]), int(r["action"][c]), int(r["obs"][c]))]
        where[c] = j
        assert r["weight"][c] == t["weight"][l][j]
        assert np.allclose(r["belief"][c], t["belief"][l][j], rtol=0, atol=1e-12)
        assert r["depth"][c] == l
    # leaf values of nodes never expanded: the upper bound of their belief
    leaves = np.flatnonzero(r["count"].sum(axis=1) == 0)
    for c in leaves[:20]:
        assert r["U"][c] == pytest.approx(O.leaf_value(w, Qu, r["belief"][c])[0], rel=1e-12)
        assert r["L"][c] == pytest.approx(O.pbvi_value(G, r["belief"][c]), rel=1e-12)


def test_one_expansion_is_the_depth_one_tree():
    w, Qu, G = _setup(2)
    r = O.bestfirst(w, Qu, G, 1)
    t = O.tree_plan(w, Qu, depth=1, K=w.K, store_levels=1)
    assert r["nodes"] == 1 + int(t["n_level"][1])
    assert np.allclose(r["UQ"][0], t["UQ"][0][0], rtol=0, atol=1e-10)
    assert np.allclose(r["R"][0], t["R"][0][0], rtol=0, atol=1e-12)
    b = O.tree_bounds(t, O.pbvi_value(G, t["belief"][1]), w.discount)
    assert np.allclose(r["LQ"][0], b["LQ"][0][0], rtol=0, atol=1e-10)
    assert r["L"][0] == pytest.approx(b["LV"][0][0], rel=1e-12)
    assert r["H"][0] == pytest.approx(b["HV"][0][0], rel=1e-12)
    assert r["E"][0] == 1 + int(b["EV"][0][0])


@pytest.mark.parametrize("seed", [3, 4])
def test_each_iteration_expands_the_root_pointer(seed):
    w, Qu, G = _setup(seed)
    full = O.bestfirst(w, Qu, G, 12, max_depth=5)
    for t in range(1, 12):
        if full["expanded"][t] < 0:
            break
        part = O.bestfirst(w, Qu, G, t, max_depth=5)
        assert full["expanded"][t] == part["E"][0]


@pytest.mark.parametrize("seed", [5, 6])
def test_root_pointer_path_and_bounds(seed):
    w, Qu, G = _setup(seed)
    r = O.bestfirst(w, Qu, G, 15, max_depth=6)
    assert np.all(r["L"] <= r["U"] + 1e-9)
    closed = r["depth"] >= 6
    assert np.all(r["H"][closed] == 0.0)
    # walk down from the root along Eq. 9's choices
    v, prod = 0, 1.0
    while r["count"][v].sum() > 0:
        a = int(np.argmax(r["UQ"][v]))
        c0, n = int(r["first"][v, a]), int(r["count"][v, a])
        ch = np.arange(c0, c0 + n)
        h = w.discount * r["weight"][ch] * r["H"][ch]
        c = int(ch[int(np.argmax(h))])
        prod *= w.discount * r["weight"][c]
        v = c
    assert v == r["E"][0]
    gap = r["U"][v] - r["L"][v] if r["depth"][v] < 6 else 0.0
    assert r["H"][0] == pytest.approx(prod * gap, rel=1e-12, abs=1e-15)


def _path_margin(r, gamma):
    """The gaps of the comparisons from the root down the pointer path, from
    the fields of a finished run (numpy, independent of the C loop)."""
    m, u = np.inf, 0
    while r["count"][u].sum() > 0:
        uq = r["UQ"][u]
        au = int(np.argmax(uq))
        m = min(m, min((uq[au] - uq[a] for a in range(5) if a != au), default=np.inf))
        c0, n = int(r["first"][u][au]), int(r["count"][u][au])
        ch = np.arange(c0, c0 + n)
        h = gamma * r["weight"][ch] * r["H"][ch]
        k = int(np.argmax(h))
        if n > 1:
            m = min(m, float(h[k] - np.delete(h, k).max()))
        u = int(ch[k])
    return m


def test_margin_is_the_smallest_gap_on_the_pointer_path():
    # margin[t] is taken on the tree of the first t expansions: recompute it
    # from the fields of a run stopped after t iterations
    w, Qu, G = _setup(7)
    full = O.bestfirst(w, Qu, G, 7, max_depth=5)
    assert full["margin"][0] == np.inf and np.all(full["margin"][:full["iterations"]] >= 0.0)
    for t in range(1, 7):
        r = O.bestfirst(w, Qu, G, t, max_depth=5)
        assert full["margin"][t] == pytest.approx(_path_margin(r, w.discount), rel=1e-12, abs=1e-12), t
        assert full["expanded"][t] == r["E"][0]
