"""Pins for the oracle of the paper's experimental model (Sec. V): nine
actions, four occupancy sensors, the paper's stage reward.  The oracle's
per-cell rows are checked against the dense brute force of `brute9` (whole-
grid shifts, a separate formulation of the same reading), its value
iteration against the dense iteration and an exact policy-evaluation solve,
its Bayes update against dense products, its tree against a dense tree
and the closed form that holds with exact motion and exact sensors, and its
value iteration on a corridor against the closed form of a walk to the
goal.  None of these call the CUDA library."""
import numpy as np
import pytest

import oracle as O
from paper_1810_00204_gb300 import workloads as WL

import brute9 as B9


def _w(seed=0, H=9, W=11, **kw):
    w = WL.tiny(seed, H=H, W=W)
    for k, v in kw.items():
        setattr(w, k, v)
    return w


def _dense_rows(w):
    n = w.H * w.W
    T = np.zeros((9, n, n))
    for a in range(9):
        for x in range(n):
            for y, p in O.transition_row9(w, x, a).items():
                T[a, x, y] += p
    return T


@pytest.mark.parametrize("seed", [0, 3])
def test_transition_rows_match_dense_model(seed):
    w = _w(seed)
    T = _dense_rows(w)
    Tb = B9.dense_T(w)
    assert np.abs(T - Tb).max() <= 1e-15
    assert np.allclose(T.sum(axis=2), 1.0, atol=1e-15)


def test_tprime_reading_on_open_ground():
    # an interior cell with a free 3x3 neighbourhood: the move gets 1 - 2 eps,
    # the two cells 45 degrees off get eps each, stay keeps the cell
    H, W = 7, 7
    occ = np.zeros((H, W), np.uint8)
    w = WL.custom(H, W, occ, np.array([0], np.int32), 1, 0, 24, 0.1, 0.9, 0.95,
                  np.full((H, W), 1.0 / 49, np.float32))
    eps = w.slip
    x = 3 * W + 3
    up = O.transition_row9(w, x, 1)
    assert up == pytest.approx({2 * W + 3: 1 - 2 * eps, 2 * W + 4: eps, 2 * W + 2: eps})
    diag = O.transition_row9(w, x, 8)  # down-right: slips to right and down
    assert diag == pytest.approx({4 * W + 4: 1 - 2 * eps, 3 * W + 4: eps, 4 * W + 3: eps})
    assert O.transition_row9(w, x, 4) == {x: 1.0}
    # a wall above folds the intended move and its slips back onto x
    occ[2, 2:5] = 1
    w.occ = occ
    assert O.transition_row9(w, x, 1) == pytest.approx({x: 1.0})
    # the grid's edge acts as a wall
    assert O.transition_row9(w, 0 * W + 3, 1) == pytest.approx({3: 1.0})


@pytest.mark.parametrize("seed", [0, 5])
def test_rewards_match_dense_model(seed):
    w = _w(seed)
    assert np.abs(O.reward_table9(w) - B9.dense_R(w)).max() <= 1e-15


def test_reward_closed_forms():
    H, W = 7, 7
    occ = np.zeros((H, W), np.uint8)
    occ[1, 3] = 1
    w = WL.custom(H, W, occ, np.array([0], np.int32), 1, 6 * W + 6, 24, 0.1, 0.9, 0.95,
                  np.full((H, W), 1.0 / 48, np.float32))
    eps = w.slip
    R = O.reward_table9(w)
    x = 4 * W + 3
    assert R[1, x] == pytest.approx(-1.0) and R[4, x] == -2.0
    # moving up from (2, 3) aims at the wall: -2 (1 - 2 eps) - eps - eps
    assert R[1, 2 * W + 3] == pytest.approx(-2 * (1 - 2 * eps) - 2 * eps)
    # onto the goal from (5, 6): 0 (1 - 2 eps), one slip free (-1), one outside (-2)
    assert R[7, 5 * W + 6] == pytest.approx(-eps - 2 * eps)
    assert np.all(R[:, w.goal] == 0.0)


@pytest.mark.parametrize("seed", [0, 2])
def test_sensor_model(seed):
    w = _w(seed)
    n = w.H * w.W
    Od = B9.dense_O(w)
    Oo = np.array([[O.obs_lik9(w, x, z) for z in range(16)] for x in range(n)])
    assert np.abs(Oo - Od).max() <= 1e-15
    assert np.allclose(Oo.sum(axis=1), 1.0, atol=1e-14)
    # the corner (0, 0) has the outside above and to the left: sensors 0, 1
    assert O.pattern9(w, 0) & 3 == 3
    assert O.obs_lik9(w, 0, O.pattern9(w, 0)) == pytest.approx(w.p_sensor ** 4)


@pytest.mark.parametrize("seed", [0, 1])
def test_value_iteration_sweeps_match_dense(seed):
    w = _w(seed)
    for k in (1, 7, 40):
        o = O.value_iteration9(w, truncated=k)
        V, Q, _ = B9.value_iteration(w, sweeps=k)
        assert np.abs(o["V"] - V).max() <= 1e-10
        assert np.abs(o["Q"] - Q).max() <= 1e-10


def test_value_iteration_is_the_greedy_policys_value():
    w = _w(4)
    o = O.value_iteration9(w, tol=1e-12)
    assert o["converged"]
    T, R = B9.dense_T(w), B9.dense_R(w)
    n = w.H * w.W
    pi = o["Q"].argmax(axis=0)
    Tp = T[pi, np.arange(n)]
    Rp = R[pi, np.arange(n)]
    Vp = np.linalg.solve(np.eye(n) - w.discount * Tp, Rp)
    live = (w.occ.ravel() == 0)
    live[w.goal] = False
    assert np.abs(o["V"][live] - Vp[live]).max() <= 1e-9


@pytest.mark.parametrize("seed", [0, 3])
def test_bayes_update_matches_dense(seed):
    w = _w(seed)
    rng = np.random.default_rng(seed)
    b = rng.random(w.H * w.W) * (w.occ.ravel() == 0)
    b /= b.sum()
    T, Od = B9.dense_T(w), B9.dense_O(w)
    for a in (0, 1, 4, 8):
        bbar = O.predict9(w, b, a)
        assert np.abs(bbar - b @ T[a]).max() <= 1e-15
        assert bbar.sum() == pytest.approx(1.0, abs=1e-13)
        P = O.obs_marginal9(w, bbar)
        assert np.abs(P - bbar @ Od).max() <= 1e-15 and P.sum() == pytest.approx(1.0, abs=1e-13)
        for z in (0, 5, 15):
            bz, pz = O.correct9(w, bbar, z)
            assert pz == pytest.approx(P[z], rel=1e-13)
            assert np.abs(bz - Od[:, z] * bbar / P[z]).max() <= 1e-13


def test_uninformative_sensors_leave_the_prediction():
    w = _w(1, p_sensor=0.5)
    b = w.b0.ravel().astype(np.float64)
    bbar = O.predict9(w, b, 2)
    assert np.allclose(O.obs_marginal9(w, bbar), 1.0 / 16, atol=1e-15)
    bz, _ = O.correct9(w, bbar, 9)
    assert np.abs(bz - bbar / bbar.sum()).max() <= 1e-15


def _dense_tree(w, Q, depth, K):
    """The sampled tree with dense matrices; samples from the oracle's
    uniform stream and an FP32 inverse CDF written here."""
    T, Od, R = B9.dense_T(w), B9.dense_O(w), B9.dense_R(w)
    L = O.lib()

    def sample(P, u):
        C = np.cumsum(P.astype(np.float32), dtype=np.float32)
        t = np.float32(u) * C[-1]
        hit = np.flatnonzero(t < C)
        return int(hit[0]) if len(hit) else len(P) - 1

    def node(b, l, code):
        if l == depth:
            return (Q @ b).max()
        best = -np.inf
        qs = []
        for a in range(9):
            bbar = b @ T[a]
            P = bbar @ Od
            path = code * 9 + a
            zs = [sample(P, L.or_uniform(w.seed, w.episode, l, path, k)) for k in range(K)]
            s = 0.0
            for z in sorted(set(zs)):
                child = Od[:, z] * bbar / P[z]
                s += zs.count(z) / K * node(child, l + 1, path * 16 + z)
            q = b @ R[a] + w.discount * s
            qs.append(q)
            best = max(best, q)
        return best if l > 0 else (best, qs)

    b0 = w.b0.ravel().astype(np.float64) * (w.occ.ravel() == 0)
    return node(b0, 0, 0)


@pytest.mark.parametrize("seed", [0, 2])
def test_tree_matches_dense_tree(seed):
    w = _w(seed, H=7, W=8)
    Q = O.value_iteration9(w)["Q"]
    t = O.tree_plan9(w, Q, depth=2, K=3)
    assert t["boundary_count"] == 0
    v, qs = _dense_tree(w, Q, 2, 3)
    assert t["root_value"] == pytest.approx(v, rel=1e-12)
    assert np.allclose(t["root_q"], qs, rtol=1e-12, atol=1e-12)


def test_exact_motion_and_sensors_give_the_mdp_value():
    # eps = 0, p_sensor = 1 and a one-cell b0: every action has one child,
    # and the tree's value is the optimal value of the start cell
    w = _w(3, H=9, W=9, slip=0.0, p_sensor=1.0)
    b0 = np.zeros((w.H, w.W), np.float32)
    b0.ravel()[w.start] = 1.0
    w.b0 = b0
    o = O.value_iteration9(w, tol=1e-13)
    for d in (1, 2, 3):
        t = O.tree_plan9(w, o["Q"], depth=d, K=2)
        assert list(t["n_level"]) == [9 ** l for l in range(d + 1)]
        assert t["root_value"] == pytest.approx(o["V"][w.start], abs=1e-9)
        assert t["root_q"][t["root_action"]] == pytest.approx(o["Q"][:, w.start].max(), abs=1e-9)


def test_corridor_closed_form():
    # one row, no slip, the goal at the east end: the best policy steps east
    # (-1 per step, 0 for the step onto the goal), so a cell d steps away has
    # V = -(1 - gamma^(d-1)) / (1 - gamma); every other move costs at least
    # as much (into the outside: -2, staying: -2)
    H, W = 1, 9
    occ = np.zeros((H, W), np.uint8)
    goal = W - 1
    b0 = np.zeros((H, W), np.float32)
    b0[0, 0] = 1.0
    w = WL.custom(H, W, occ, np.array([0], np.int32), 1, goal, 0, 0.0, 0.9, 0.9, b0)
    o = O.value_iteration9(w, tol=1e-14)
    g = w.discount
    for c in range(W - 1):
        d = goal - c
        assert o["V"][c] == pytest.approx(-(1 - g ** (d - 1)) / (1 - g), abs=1e-10), c
    assert o["V"][goal] == 0.0
    assert int(np.argmax(o["Q"][:, 0])) == 5   # east
