"""Pins for the oracle's best-first QV-Tree Search (Alg. 1's planning loop
with Alg. 2-7 and Eq. 9): every node it creates is the node of the same
path in the level-synchronous tree (same samples, belief, weight and leaf
value); one expansion of the root is the depth-1 level-synchronous tree with
its AEMS fields; each iteration expands the root's E of the tree before it;
the root's E is reached by the greedy actions and the largest gamma w H_V
children, with the root's H the product along that path; lower bounds stay
below upper bounds; nodes at the depth limit are closed.  None of these call
the CUDA library."""
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


def test_forcing_its_own_choices_changes_nothing():
    w, Qu, G = _setup(7)
    r = O.bestfirst(w, Qu, G, 14, max_depth=5)
    f = O.bestfirst(w, Qu, G, 14, max_depth=5, force=r["expanded"])
    assert f["nodes"] == r["nodes"] and np.array_equal(f["expanded"], r["expanded"])
    assert np.array_equal(f["U"], r["U"]) and np.array_equal(f["E"], r["E"])
    it = r["iterations"]
    assert np.array_equal(f["forced_h"][:it], f["best_h"][:it])
    assert np.all(f["slack"][:it] == 0.0)
    # any other leaf either scores below the root's H along greedy actions or
    # hangs under a non-greedy action (a positive U_Q shortfall)
    for leaf in range(1, r["count"][0].sum() + 1):
        g = O.bestfirst(w, Qu, G, 2, max_depth=5, force=[0, leaf])
        assert g["forced_h"][1] <= g["best_h"][1] or g["slack"][1] > 0.0
        if leaf != r["expanded"][1]:
            assert g["forced_h"][1] < g["best_h"][1] or g["slack"][1] > 0.0
