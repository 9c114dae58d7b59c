"""Pins for the oracle's point-based value iteration (Sec. IV-B, Eq. 8) and
its belief set expansion: the point-based backup equals the exact Bellman
backup (brute-force expectimax over every observation, dense matrices) at
its own point; with an exact sensor and every corner belief in the set it
converges to the MDP values; its values stay below the FIB upper bound and
below an exact backup of it; the pessimistic start is below its first
backup; expanded points are tau(b, a, z) of their parents, with a uniform
action and z drawn from P(z | b, a).  None of these call the CUDA library."""
import numpy as np
import pytest

import oracle as O
from paper_1810_00204_gb300 import workloads as WL

import brute


def _w(seed, H=6, W=7, **kw):
    w = WL.tiny(seed, H=H, W=W, depth=1, K=4)
    for k, v in kw.items():
        setattr(w, k, v)
    return w


def _dead(w):
    d = w.occ.ravel().astype(bool).copy()
    d[w.goal] = True
    return d


def _rand_beliefs(w, m, seed):
    rng = np.random.default_rng(seed)
    free = np.flatnonzero(w.occ.ravel() == 0)
    out = np.zeros((m, w.H * w.W))
    for j in range(m):
        idx = rng.choice(free, size=1 + j % min(len(free), 6), replace=False)
        out[j, idx] = rng.random(len(idx))
        out[j] /= out[j].sum()
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_backup_is_the_exact_bellman_backup_at_its_point(seed):
    # Eq. 8 at b equals (H V_Gamma)(b) with V_Gamma(b') = max_alpha alpha . b'
    w = _w(seed)
    w.cost = None
    rng = np.random.default_rng([3, seed])
    G = rng.normal(-5.0, 20.0, (4, w.H * w.W))
    G[:, _dead(w)] = 0.0
    B = _rand_beliefs(w, 5, seed)
    bk = O.pbvi_backup(w, B, G)
    for j in range(len(B)):
        want = brute.expectimax(w, G, B[j], 1)
        assert bk["value"][j] == pytest.approx(want, rel=1e-10, abs=1e-9)
        # the new vector evaluated at its own point gives that value
        assert bk["G"][j] @ B[j] == pytest.approx(bk["value"][j], rel=1e-10, abs=1e-9)
        assert np.all(bk["G"][j][_dead(w)] == 0.0)


def _perfect_sensing(seed):
    rng = np.random.default_rng([21, seed])
    H, W = 4, 5
    occ = (rng.random((H, W)) < 0.2).astype(np.uint8)
    free = np.flatnonzero(occ.ravel() == 0)
    b0 = np.zeros(H * W)
    b0[free[-1]] = 1.0
    return WL.custom(H, W, occ, free, 0, int(free[0]), int(free[-1]), 0.15, 1.0, 0.9, b0)


@pytest.mark.parametrize("seed", [0, 1])
def test_corner_beliefs_with_an_exact_sensor_converge_to_mdp_values(seed):
    # every cell has its own label and the sensor is exact, so tau maps a
    # corner belief to a corner belief: a set holding every corner is closed
    # under the belief update and PBVI on it is exact value iteration
    w = _perfect_sensing(seed)
    n = w.H * w.W
    cells = np.flatnonzero(~_dead(w))
    B = np.eye(n)[cells]
    G = O.pbvi_init(w)[None, :]
    for _ in range(350):
        G = O.pbvi_backup(w, B, G)["G"]
    V = O.value_iteration(w, tol=1e-13)["V"]
    assert np.allclose(O.pbvi_value(G, B), V[cells], rtol=0, atol=1e-7)


@pytest.mark.parametrize("seed", [0, 3])
def test_pbvi_stays_below_the_upper_bounds(seed):
    w = _w(seed, H=5, W=6)
    w.cost = None
    r = O.pbvi_solve(w, rounds=3, iters=25)
    f = O.fib_iteration(w, tol=1e-12)["alpha"]
    pts = np.concatenate([r["B"], _rand_beliefs(w, 6, seed)])
    for b in pts:
        v = O.pbvi_value(r["G"], b)
        v_fib, _ = O.leaf_value(w, f, b)
        assert v <= v_fib + 1e-9
        # an exact backup of the upper bound is still an upper bound
        assert v <= brute.expectimax(w, f, b, 1) + 1e-9


def test_pessimistic_start_is_below_its_backup():
    w = _w(4)
    a0 = O.pbvi_init(w)
    R = O.reward_table(w)
    live = ~_dead(w)
    assert np.allclose(a0[live], R[:, live].min() / (1 - w.discount))
    assert np.all(a0[~live] == 0.0)
    B = _rand_beliefs(w, 6, 4)
    bk = O.pbvi_backup(w, B, a0[None, :])
    assert np.all(bk["value"] >= B @ a0 - 1e-12)


def test_expanded_points_are_tau_of_their_parents():
    w = _w(5)
    T = brute.dense_T(w)
    Om = brute.dense_O(w)
    B = _rand_beliefs(w, 7, 5)
    e = O.pbvi_expand(w, B, 2, seed=11)
    for j in range(len(B)):
        a, z = int(e["action"][j]), int(e["obs"][j])
        assert 0 <= a < 5 and 0 <= z <= w.B
        bbar = T[a].T @ B[j]
        pz = Om[:, z] @ bbar
        assert pz > 0
        assert np.allclose(e["points"][j], Om[:, z] * bbar / pz, rtol=0, atol=1e-12)
    assert np.allclose(e["points"].sum(axis=1), 1.0)
    assert np.all(e["points"][:, w.occ.ravel() == 1] == 0.0)
    # the draws are a function of (seed, round, point index) alone
    e2 = O.pbvi_expand(w, B, 2, seed=11)
    assert np.array_equal(e["obs"], e2["obs"]) and np.array_equal(e["action"], e2["action"])
    e3 = O.pbvi_expand(w, B, 3, seed=11)
    assert not np.array_equal(e["action"], e3["action"])


def test_expansion_draws_follow_their_laws():
    # 4000 expansions of one belief: the action is uniform over the five, and
    # for every action the observation follows P(z | b, a) (chi-square tests
    # at the 1e-4 level)
    from scipy.stats import chisquare
    w = _w(6, H=8, W=8)
    free = np.flatnonzero(w.occ.ravel() == 0)
    b = np.zeros(w.H * w.W)
    b[free] = 1.0 / len(free)
    B = np.repeat(b[None, :], 4000, axis=0)
    e = O.pbvi_expand(w, B, 0, seed=5)
    cnt = np.bincount(e["action"], minlength=5)
    assert chisquare(cnt).pvalue > 1e-4
    T = brute.dense_T(w)
    Om = brute.dense_O(w)
    for a in range(5):
        zs = e["obs"][e["action"] == a]
        P = Om.T @ (T[a].T @ b)
        keep = P * len(zs) >= 5
        obs = np.bincount(zs, minlength=w.B + 1)
        f_obs = np.append(obs[keep], obs[~keep].sum())
        f_exp = np.append(P[keep], P[~keep].sum()) * len(zs)
        if f_exp[-1] == 0:
            f_obs, f_exp = f_obs[:-1], f_exp[:-1]
        assert chisquare(f_obs, f_exp).pvalue > 1e-4
