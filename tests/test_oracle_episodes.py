"""Pins for the oracle's closed-loop episodes (Alg. 1's outer loop, Eq. 1):
the true system's motion and measurement draws follow T (Sec. II, Eq. 10)
and O (chi-square), blocked moves and the goal stay; every step of a
recorded episode is the plan of the belief rebuilt from b0 and the recorded
(action, measurement) pairs, and the recorded state the system's step;
success, steps and the discounted return follow from the states; with no
slip and an exact sensor naming every cell, the loop walks a shortest path.
None of these call the CUDA library."""
from collections import deque

import numpy as np
import pytest
from scipy.stats import chisquare

import oracle as O
from paper_1810_00204_gb300 import workloads as WL

import brute


def test_motion_and_measurement_laws():
    w = WL.tiny(2, H=9, W=10)
    T = brute.dense_T(w)
    Om = brute.dense_O(w)
    free = np.flatnonzero(w.occ.ravel() == 0)
    x = int(free[len(free) // 2])
    if x == w.goal:
        x = int(free[len(free) // 2 + 1])
    for a in range(5):
        ys, zs = [], []
        for step in range(3000):
            y, z = O.env_step(w, x, a, seed=9, e=3, step=step)
            ys.append(y)
            zs.append(z)
        ys, zs = np.array(ys), np.array(zs)
        support = np.flatnonzero(T[a][x] > 0)
        assert set(np.unique(ys)) <= set(support)
        if len(support) > 1:
            f_obs = np.array([(ys == y).sum() for y in support])
            assert chisquare(f_obs, T[a][x][support] * len(ys)).pvalue > 1e-4
        # the measurement at the reached cell
        for y in np.unique(ys)[:1]:
            zz = zs[ys == y]
            P = Om[y]
            keep = P * len(zz) >= 5
            f_obs = np.bincount(zz, minlength=w.B + 1)
            fo = np.append(f_obs[keep], f_obs[~keep].sum())
            fe = np.append(P[keep], P[~keep].sum()) * len(zz)
            if fe[-1] == 0:
                fo, fe = fo[:-1], fe[:-1]
            assert chisquare(fo, fe).pvalue > 1e-4
    # the goal and the stay action keep the state
    assert O.env_step(w, w.goal, 1, 9, 0, 0)[0] == w.goal
    assert O.env_step(w, x, 4, 9, 0, 5)[0] == x


def _episodes(seed, E=6, S=40, **over):
    w = WL.tiny(seed, H=12, W=13, depth=2, K=4)
    for k, v in over.items():
        setattr(w, k, v)
    eps = WL.episodes(w, E, seed=seed)
    Q = O.value_iteration(w)["Q"]
    r = O.closed_loop(w, Q, [e.b0 for e in eps], [e.start for e in eps], max_steps=S)
    return w, eps, Q, r


@pytest.mark.parametrize("seed", [0, 1])
def test_every_step_is_the_plan_of_the_rebuilt_belief(seed):
    w, eps, Q, r = _episodes(seed)
    E = len(eps)
    lab = O.labels(w)
    for e in range(E):
        b = eps[e].b0.ravel().astype(np.float64)
        x = eps[e].start
        for t in range(r["steps"][e]):
            tr = O.tree_plan(w, Q, b0=b, episode=t * E + e)
            a = r["actions"][e, t]
            assert a == tr["root_action"]
            y, z = O.env_step(w, x, a, w.seed, e, t)
            assert (y, z) == (r["states"][e, t + 1], r["obs"][e, t])
            b, _ = O.correct(w, O.predict(w, b, a), z, lab)
            x = y


@pytest.mark.parametrize("seed", [2, 3])
def test_outcomes_follow_from_the_states(seed):
    w, eps, Q, r = _episodes(seed)
    for e in range(len(eps)):
        n = r["steps"][e]
        st = r["states"][e, :n + 1]
        assert r["success"][e] == int(st[-1] == w.goal)
        assert np.all(st[:-1] != w.goal)
        assert np.all(r["states"][e, n + 1:] == -1) and np.all(r["actions"][e, n:] == -1)
        rew = np.where(st[1:] == w.goal, 100.0, -1.0 - (0.0 if w.cost is None else w.cost.ravel()[st[1:]]))
        assert r["ret"][e] == pytest.approx(np.sum(rew * w.discount ** np.arange(n)), rel=1e-12)


def _bfs(occ, W, s):
    """Shortest-path lengths from s over the free cells (4-connected)."""
    H = occ.size // W
    dist = {s: 0}
    q = deque([s])
    while q:
        u = q.popleft()
        r, c = divmod(u, W)
        for dr, dc in ((-1, 0), (0, 1), (1, 0), (0, -1)):
            rr, cc = r + dr, c + dc
            if 0 <= rr < H and 0 <= cc < W and not occ[rr * W + cc] and rr * W + cc not in dist:
                dist[rr * W + cc] = dist[u] + 1
                q.append(rr * W + cc)
    return dist


def test_exact_sensing_without_slip_walks_a_shortest_path():
    H, W = 7, 8
    w0 = WL.tiny(0, H=H, W=W)
    occ = w0.occ.copy()
    free = np.flatnonzero(occ.ravel() == 0)
    goal = int(w0.goal)
    dist = _bfs(occ.ravel(), W, goal)
    starts = [int(s) for s in free if s != goal and s in dist][:6]
    assert len(starts) == 6
    b0s = np.zeros((len(starts), H * W))
    for i, s in enumerate(starts):
        b0s[i, s] = 1.0
    w = WL.custom(H, W, occ, free, 0, goal, starts[0], 0.0, 1.0, 0.95, b0s[0], depth=1, K=1)
    Q = O.value_iteration(w, tol=1e-12)["Q"]
    r = O.closed_loop(w, Q, b0s, starts, depth=1, K=1, max_steps=60)
    for i, s in enumerate(starts):
        assert r["success"][i] == 1
        assert r["steps"][i] == dist[s]
