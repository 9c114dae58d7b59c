"""Pins for the oracle's Fast Informed Bound (Sec. IV-A, Eq. 6-7): its
relation to the QMDP alpha-vectors (below them, equal to them when the sensor
identifies every cell), the closed form it reduces to when the sensor carries
no information, the stay action's closed form, Sec. IV-A's contraction and
monotonicity, and its being an upper bound that an exact one- or two-step
Bellman backup (brute-force expectimax over every observation) cannot raise.
None of these call the CUDA library."""
import numpy as np
import pytest

import oracle as O
from paper_1810_00204_gb300 import workloads as WL

import brute


def _w(seed, H=7, W=8, **kw):
    w = WL.tiny(seed, H=H, W=W, depth=1, K=4)
    for k, v in kw.items():
        setattr(w, k, v)
    return w


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_fib_is_below_qmdp(seed):
    w = _w(seed)
    f = O.fib_iteration(w, tol=1e-12)
    v = O.value_iteration(w, tol=1e-12)
    assert f["converged"] and v["converged"]
    assert np.all(f["alpha"] <= v["Q"] + 1e-9)
    # a partially informative sensor makes the bound strictly tighter somewhere
    assert (v["Q"] - f["alpha"]).max() > 1e-3


def _perfect_sensing(seed):
    rng = np.random.default_rng([11, seed])
    H, W = 5, 6
    occ = (rng.random((H, W)) < 0.2).astype(np.uint8)
    free = np.flatnonzero(occ.ravel() == 0)
    goal = int(free[0])
    b0 = np.zeros(H * W)
    b0[free[-1]] = 1.0
    # one beacon on every free cell with range 0: each free cell has a label of its own
    return WL.custom(H, W, occ, free, 0, goal, int(free[-1]), 0.15, 1.0, 0.93, b0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fib_equals_qmdp_when_the_sensor_names_the_cell(seed):
    # O(x', z) = 1[z = label(x')] with distinct labels: the max over a' moves
    # inside the sum over x', and Eq. 7 becomes the MDP Bellman equation on Q.
    w = _perfect_sensing(seed)
    f = O.fib_iteration(w, tol=1e-12)
    v = O.value_iteration(w, tol=1e-12)
    assert np.allclose(f["alpha"], v["Q"], rtol=0, atol=1e-9)


@pytest.mark.parametrize("seed", [0, 4])
def test_fib_with_an_uninformative_sensor(seed):
    # alpha = eta = 1/(B+1): O(x', z) = 1/|Z| for every pair, so Eq. 7 reduces to
    #   alpha^a(x) = R(x, a) + gamma max_a' sum_x' T(x, a, x') alpha^a'(x'),
    # solved here with dense matrices built independently of the oracle.
    w = _w(seed)
    w.accuracy = 1.0 / (w.B + 1)
    T = brute.dense_T(w)
    R = brute.dense_R(w, T, w.cost)
    dead = w.occ.ravel().astype(bool).copy()
    dead[w.goal] = True
    al = np.zeros((5, w.H * w.W))
    for _ in range(5000):
        nxt = R + w.discount * np.einsum("axy,by->abx", T, al).max(axis=1)
        nxt[:, dead] = 0.0
        if np.abs(nxt - al).max() < 1e-13:
            al = nxt
            break
        al = nxt
    f = O.fib_iteration(w, tol=1e-13)
    assert np.allclose(f["alpha"], al, rtol=0, atol=1e-8)


def test_stay_action_closed_form():
    # Staying keeps the state, and sum_z O(x, z) = alpha + B eta = 1, so one
    # application of Eq. 7 gives alpha'^4(x) = R(x, 4) + gamma max_a' alpha^a'(x)
    # for any input alpha.
    w = _w(5)
    rng = np.random.default_rng(5)
    al = rng.normal(0, 10, (5, w.H * w.W))
    out, _ = O.fib_sweep(w, al)
    R = O.reward_table(w)
    dead = w.occ.ravel().astype(bool).copy()
    dead[w.goal] = True
    want = np.where(dead, 0.0, R[4] + w.discount * al.max(axis=0))
    assert np.allclose(out[4], want, rtol=0, atol=1e-10)


def test_contraction_and_monotonicity():
    w = _w(6)
    f = O.fib_iteration(w, tol=1e-12)
    h = f["hist"]
    # |alpha_{k+2} - alpha_{k+1}| <= gamma |alpha_{k+1} - alpha_k| (sup norm)
    assert np.all(h[1:] <= w.discount * h[:-1] * (1 + 1e-9) + 1e-12)
    rng = np.random.default_rng(6)
    a = rng.normal(0, 20, (5, w.H * w.W))
    b = a + np.abs(rng.normal(0, 5, a.shape))
    ha, _ = O.fib_sweep(w, a)
    hb, _ = O.fib_sweep(w, b)
    assert np.all(ha <= hb + 1e-10)
    # sup-norm contraction of the operator itself
    assert np.abs(hb - ha).max() <= w.discount * np.abs(b - a).max() + 1e-10


@pytest.mark.parametrize("seed,depth", [(0, 1), (1, 1), (2, 2)])
def test_exact_backups_do_not_raise_the_bound(seed, depth):
    # V_FIB is the fixed point of an operator that bounds the exact Bellman
    # operator from above, so H^d V_FIB(b) <= V_FIB(b) for every belief b;
    # the exact backups enumerate every observation (Eq. 2).
    w = _w(seed, H=5, W=6)
    w.cost = None
    f = O.fib_iteration(w, tol=1e-13)
    Qm = O.value_iteration(w, tol=1e-13)["Q"]
    rng = np.random.default_rng([9, seed])
    free = np.flatnonzero(w.occ.ravel() == 0)
    for t in range(6):
        b = np.zeros(w.H * w.W)
        idx = rng.choice(free, size=min(len(free), 1 + t * 3), replace=False)
        b[idx] = rng.random(len(idx))
        b /= b.sum()
        v_fib, _ = O.leaf_value(w, f["alpha"], b)
        v_qmdp, _ = O.leaf_value(w, Qm, b)
        assert v_fib <= v_qmdp + 1e-9
        assert brute.expectimax(w, f["alpha"], b, depth) <= v_fib + 1e-8


def test_one_sweep_matches_dense_matrices():
    # the sparse transition rows and per-cell labels against dense T and O
    w = _w(7)
    T = brute.dense_T(w)
    Om = brute.dense_O(w)
    R = brute.dense_R(w, T, w.cost)
    dead = w.occ.ravel().astype(bool).copy()
    dead[w.goal] = True
    rng = np.random.default_rng(7)
    al = rng.normal(0, 10, (5, w.H * w.W))
    # s[a, b, z, x] = sum_x' T[a, x, x'] O[x', z] al[b, x']
    s = np.einsum("axy,yz,by->abzx", T, Om, al)
    want = R + w.discount * s.max(axis=1).sum(axis=1)
    want[:, dead] = 0.0
    out, _ = O.fib_sweep(w, al)
    assert np.allclose(out, want, rtol=0, atol=1e-9)
