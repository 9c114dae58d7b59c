"""Pins for the oracle's AEMS bookkeeping over a tree (Alg. 5-7, Eq. 9):
equal bounds at the leaves give equal bounds everywhere and no heuristic;
ordered leaf bounds stay ordered; the pointer E of the root leads down the
greedy actions of U_Q and the children of largest gamma w H_V, and the root
heuristic is the product of gamma w along that path times the leaf's gap;
with every observation in the tree and exact weights the root's lower bound
is the exact depth-d expectimax (dense matrices) of V_PBVI.  None of these
call the CUDA library."""
import numpy as np
import pytest

import oracle as O
from paper_1810_00204_gb300 import workloads as WL

import brute


def _tree(seed, depth=2, K=4, weight_mode=O.FREQ, H=9, W=10):
    w = WL.tiny(seed, H=H, W=W, depth=depth, K=K)
    Q = O.fib_iteration(w)["alpha"]
    t = O.tree_plan(w, Q, depth=depth, K=K, weight_mode=weight_mode, store_levels=depth)
    return w, Q, t


@pytest.mark.parametrize("seed", [0, 1])
def test_equal_leaf_bounds_propagate(seed):
    w, Q, t = _tree(seed)
    d = t["depth"]
    b = O.tree_bounds(t, t["value"][d], w.discount)
    for l in range(d + 1):
        assert np.allclose(b["LV"][l], t["value"][l], rtol=0, atol=1e-9)
        assert np.all(b["HV"][l] == 0.0)
        if l < d:
            assert np.allclose(b["LQ"][l], t["UQ"][l], rtol=0, atol=1e-9)


@pytest.mark.parametrize("seed", [2, 3])
def test_ordered_leaf_bounds_stay_ordered(seed):
    w, Q, t = _tree(seed, depth=3, K=3)
    d = t["depth"]
    rng = np.random.default_rng(seed)
    L = t["value"][d] - rng.uniform(0.0, 5.0, len(t["value"][d]))
    b = O.tree_bounds(t, L, w.discount)
    for l in range(d + 1):
        assert np.all(b["LV"][l] <= t["value"][l] + 1e-12)
        assert np.all(b["HV"][l] >= 0.0)


@pytest.mark.parametrize("seed,depth", [(4, 2), (5, 3)])
def test_root_pointer_path(seed, depth):
    w, Q, t = _tree(seed, depth=depth, K=3)
    rng = np.random.default_rng(seed)
    L = t["value"][depth] - rng.uniform(0.0, 5.0, len(t["value"][depth]))
    b = O.tree_bounds(t, L, w.discount)
    e = int(b["EV"][0][0])
    assert 0 <= e < len(L)
    # walk up from the leaf; at every V-node the path takes the greedy action
    # of U_Q and at every Q-node the child of largest gamma w H_V
    prod, j = 1.0, e
    for l in range(depth, 0, -1):
        i, a = int(t["parent"][l][j]), int(t["action"][l][j])
        assert a == int(np.argmax(t["UQ"][l - 1][i]))
        sib = np.flatnonzero((t["parent"][l] == i) & (t["action"][l] == a))
        h = w.discount * t["weight"][l][sib] * b["HV"][l][sib]
        assert j == sib[int(np.argmax(h))]
        prod *= w.discount * t["weight"][l][j]
        j = i
    assert j == 0
    assert b["HV"][0][0] == pytest.approx(prod * (t["value"][depth][e] - L[e]), rel=1e-12)


def test_depth_zero_root_is_the_leaf():
    w, Q, t = _tree(6, depth=0, K=1)
    b = O.tree_bounds(t, [-3.0], w.discount)
    assert b["LV"][0][0] == -3.0
    assert b["HV"][0][0] == pytest.approx(t["value"][0][0] + 3.0)
    assert b["EV"][0][0] == 0


@pytest.mark.parametrize("seed", [0, 7])
def test_exact_weights_give_the_expectimax_of_pbvi(seed):
    # MARGINAL weights with every observation of nonzero probability drawn
    # are P(z | b, a): the lower-bound backup is then the exact depth-d
    # Bellman recursion (Eq. 2) with V_PBVI at the leaves
    # (a noisy sensor, alpha = 0.5, keeps every P(z) >= (1 - alpha) / B so that
    # 200 draws see every observation)
    w = WL.tiny(seed, H=6, W=7, depth=2, K=200)
    w.cost = None
    w.accuracy = 0.5
    G = O.pbvi_solve(w, rounds=2, iters=6)["G"]
    Q = O.fib_iteration(w)["alpha"]
    # b0 renormalised in FP64, so that sum_z P(z) = 1 to rounding and the
    # MARGINAL weights equal P(z)
    b0 = w.b0.ravel().astype(np.float64)
    b0 /= b0.sum()
    t = O.tree_plan(w, Q, depth=2, K=200, weight_mode=O.MARGINAL, store_levels=2, b0=b0)
    # every (node, action) of the internal levels saw every z with P(z) > 1e-9
    lab = O.labels(w)
    for l in range(2):
        for i in range(int(t["n_level"][l])):
            for a in range(5):
                P = O.obs_marginal(w, O.predict(w, t["belief"][l][i], a), lab)
                seen = t["obs"][l + 1][(t["parent"][l + 1] == i) & (t["action"][l + 1] == a)]
                assert set(np.flatnonzero(P > 1e-9)) <= set(seen.tolist())
    Ll = O.pbvi_value(G, t["belief"][2])
    b = O.tree_bounds(t, Ll, w.discount)
    want = brute.expectimax(w, G, b0, 2)
    assert b["LV"][0][0] == pytest.approx(want, rel=1e-10, abs=1e-10)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ties_take_the_first_child(seed):
    # a constant gap at every leaf makes gamma w H_V tie between siblings of
    # equal sample frequency; the pointer takes the first of them in the
    # (parent, action, z) order
    w, Q, t = _tree(seed, depth=2, K=4)
    d = t["depth"]
    b = O.tree_bounds(t, t["value"][d] - 1.0, w.discount)
    ties = 0
    for l in range(d):
        for i in range(int(t["n_level"][l])):
            for a in range(5):
                sib = np.flatnonzero((t["parent"][l + 1] == i) & (t["action"][l + 1] == a))
                h = w.discount * t["weight"][l + 1][sib] * b["HV"][l + 1][sib]
                first = sib[int(np.argmax(h))]
                ties += int(np.sum(h == h.max()) > 1)
                assert b["HQ"][l][i, a] == h.max()
                assert b["EQ"][l][i, a] == b["EV"][l + 1][first]
    assert ties > 0
