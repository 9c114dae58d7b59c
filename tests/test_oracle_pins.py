"""Pins for the FP64 oracle against what the paper and the mathematics fix:
hand-derived golden values, closed forms, invariants, an independent dense
brute force on tiny grids, and statistical checks of the sampler.  None of
these call the CUDA library."""
import math
import os

import numpy as np
import pytest

import brute
import oracle as O
from paper_1810_00204_gb300 import workloads as WL

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _grid(H, W, occ_cells=(), goal=0, slip=0.1, beacons=(0,), rng=3, acc=0.9, cost=None,
          b0=None, depth=1, K=4, discount=0.95):
    """A hand-made problem with exact (FP64) model parameters."""
    occ = np.zeros(H * W, np.uint8)
    for c in occ_cells:
        occ[c] = 1
    if b0 is None:
        b0 = (1 - occ) / (1 - occ).sum()
    w = WL.custom(H, W, occ, list(beacons), rng, goal, goal, slip, acc, discount, b0,
                  depth=depth, K=K, cost=cost)
    return O.Problem(w, slip=slip, accuracy=acc, discount=discount,
                     cost=None if cost is None else np.asarray(cost, np.float64))


def _lines(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.split("#")[0].strip() for ln in f if ln.split("#")[0].strip()]


# ------------------------------------------------------------------ Philox
def test_philox_known_answers():
    # Known-answer vectors published with the Random123 library (Salmon et al.)
    kat = [([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
           ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
           ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
            [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1])]
    for ctr, key, want in kat:
        assert list(O.philox(ctr, key)) == want


def test_uniform_exact_in_fp32_and_open_interval():
    for k in range(64):
        u = O.uniform(12345, 7, 2, 987654321, k)
        assert 0.0 < u < 1.0
        assert np.float32(u) == u
        m = u * 2 ** 24
        assert m == int(m) and int(m) % 2 == 1


def test_uniform_stream_uses_all_four_words():
    words = O.philox([0, 3, 99, (1 << 24) | 0], [5, 0])
    for k in range(4):
        u = O.uniform(5, 3, 1, 99, k)
        assert u == (2 * (int(words[k]) >> 9) + 1) / 2 ** 24


# ------------------------------------------------------------------ model
def test_transition_golden():
    for ln in _lines("transition_3x3.txt"):
        lhs, rhs = ln.split("->")
        case, H, W, occ, goal, src, a = lhs.split()
        occ_cells = [] if occ == "-" else [int(c) for c in occ.split(";")]
        w = _grid(int(H), int(W), occ_cells, goal=int(goal))
        got = O.transition_row(w, int(src), int(a))
        want = {int(t.split(":")[0]): float(t.split(":")[1]) for t in rhs.split()}
        assert set(got) == set(want), case
        for k in want:
            assert got[k] == pytest.approx(want[k], abs=1e-15), case


def test_labels_golden():
    for ln in _lines("labels.txt"):
        lhs, rhs = ln.split("->")
        case, H, W, rng, bc = lhs.split()
        beacons = [int(c) for c in bc.split(";")]
        w = _grid(int(H), int(W), goal=1, beacons=beacons, rng=int(rng))
        assert list(O.labels(w)) == [int(v) for v in rhs.split()], case


def test_reward_golden():
    for ln in _lines("reward_corridor.txt"):
        lhs, rhs = ln.split("->")
        f = lhs.split()
        cost = [float(v) for v in f[:3]]
        x, a = int(f[3]), int(f[4])
        w = _grid(1, 3, goal=0, cost=None if not any(cost) else cost)
        assert O.reward_table(w)[a, x] == pytest.approx(float(rhs), abs=1e-12)


def test_correct_golden():
    ln = _lines("correct_1x3.txt")
    P = [float(v) for v in ln[0].split()[1:]]
    w = _grid(1, 3, goal=2, beacons=[0], rng=0, acc=0.9)
    bbar = np.array([0.2, 0.3, 0.5])
    got_P = O.obs_marginal(w, bbar)
    assert got_P == pytest.approx(P, abs=1e-15)
    for z in range(2):
        want = [float(v) for v in ln[1 + z].split()[1:]]
        b, pz = O.correct(w, bbar, z)
        assert pz == pytest.approx(P[z], abs=1e-15)
        assert b == pytest.approx(want, abs=1e-15)


def test_transition_rows_match_dense_brute_force():
    for seed in range(4):
        w = WL.tiny(seed, H=7, W=6)
        T = brute.dense_T(w)
        for x in range(w.H * w.W):
            for a in range(5):
                row = O.transition_row(w, x, a)
                dense = np.zeros(w.H * w.W)
                for y, p in row.items():
                    dense[y] += p
                assert np.allclose(dense, T[a, x], atol=1e-15), (seed, x, a)


def test_labels_and_rewards_match_dense_brute_force():
    for seed in range(4):
        w = WL.tiny(seed, H=9, W=11)
        assert np.array_equal(O.labels(w), brute.dense_labels(w))
        assert np.allclose(O.reward_table(w), brute.dense_R(w), atol=1e-12)
    w = WL.diff(0, H=8, W=9)
    assert np.allclose(O.reward_table(w), brute.dense_R(w, cost=w.cost), atol=1e-12)


# ------------------------------------------------------------------ predict / correct
@pytest.fixture(scope="module")
def tinyw():
    return WL.tiny(1)


def _rand_belief(w, seed):
    rng = np.random.default_rng(seed)
    b = rng.random(w.H * w.W) * (1 - w.occ.ravel())
    return b / b.sum()


def test_predict_conserves_mass_and_nonneg(tinyw):
    for s in range(3):
        b = _rand_belief(tinyw, s)
        for a in range(5):
            bb = O.predict(tinyw, b, a)
            assert bb.sum() == pytest.approx(1.0, abs=1e-13)
            assert (bb >= 0).all()
            assert (bb[tinyw.occ.ravel() == 1] == 0).all()


def test_predict_stay_is_identity(tinyw):
    b = _rand_belief(tinyw, 9)
    assert np.array_equal(O.predict(tinyw, b, 4), b)


def test_predict_matches_dense(tinyw):
    T = brute.dense_T(tinyw)
    b = _rand_belief(tinyw, 4)
    for a in range(5):
        assert np.allclose(O.predict(tinyw, b, a), T[a].T @ b, atol=1e-15)


def test_obs_marginal_sums_to_one_and_floor(tinyw):
    lab = O.labels(tinyw)
    eta = (1 - tinyw.accuracy) / tinyw.B
    for s in range(3):
        bb = O.predict(tinyw, _rand_belief(tinyw, s), s % 5)
        P = O.obs_marginal(tinyw, bb, lab)
        assert P.sum() == pytest.approx(1.0, abs=1e-13)
        assert (P >= eta * bb.sum() - 1e-15).all()
        assert np.allclose(P, brute.dense_O(tinyw).T @ bb, atol=1e-15)


def test_correct_uniform_sensor_is_renormalisation():
    w0 = WL.tiny(2)
    # O(x, z) = 1/(B+1) for every x, z (exact FP64 parameter)
    w = O.Problem(w0, accuracy=1.0 / (w0.B + 1))
    bb = O.predict(w, _rand_belief(w0, 1), 2) * 0.7
    for z in range(w.B + 1):
        b, pz = O.correct(w, bb, z)
        assert np.allclose(b, bb / bb.sum(), atol=1e-15)
        assert pz == pytest.approx(0.7 / (w.B + 1), abs=1e-15)


def test_correct_perfect_sensor_restricts_to_label_region():
    w = WL.tiny(3)
    w.accuracy = 1.0
    lab = O.labels(w)
    bb = O.predict(w, _rand_belief(w, 5), 1)
    for z in range(w.B + 1):
        b, pz = O.correct(w, bb, z, lab)
        reg = lab == z
        if bb[reg].sum() == 0:
            continue
        assert pz == pytest.approx(bb[reg].sum(), abs=1e-15)
        assert np.allclose(b, np.where(reg, bb, 0) / bb[reg].sum(), atol=1e-15)


def test_correct_sums_to_one(tinyw):
    lab = O.labels(tinyw)
    bb = O.predict(tinyw, _rand_belief(tinyw, 7), 0)
    for z in range(tinyw.B + 1):
        b, _ = O.correct(tinyw, bb, z, lab)
        assert b.sum() == pytest.approx(1.0, abs=1e-13)
        assert (b >= 0).all()


# ------------------------------------------------------------------ value iteration
@pytest.mark.parametrize("eps,gamma", [(0.0, 0.9), (0.1, 0.95), (0.15, 0.97)])
def test_vi_corridor_closed_form(eps, gamma):
    L = 12
    w = _grid(1, L, goal=0, slip=eps, discount=gamma)
    vi = O.value_iteration(w, tol=1e-13, max_sweeps=100000)
    # moving toward the goal: V(d) = [(1-2e)(r_{d-1} + g V(d-1)) - 2e] / (1 - 2 e g),
    # r_0 = +100 (arrival at the goal), r_{>0} = -1; V(0) = 0
    want = [0.0]
    for d in range(1, L):
        r = 100.0 if d == 1 else -1.0
        want.append(((1 - 2 * eps) * (r + gamma * want[-1]) - 2 * eps) / (1 - 2 * eps * gamma))
    assert np.allclose(vi["V"], want, atol=1e-10)
    if eps == 0.0:
        for d in range(1, L):
            closed = -(1 - gamma ** (d - 1)) / (1 - gamma) + 100 * gamma ** (d - 1)
            assert vi["V"][d] == pytest.approx(closed, abs=1e-10)


def test_vi_contraction(tinyw):
    vi = O.value_iteration(tinyw, tol=1e-10)
    h = vi["hist"]
    assert vi["converged"]
    assert (h[1:] <= tinyw.discount * h[:-1] * (1 + 1e-12) + 1e-14).all()


def test_vi_fixed_point_is_policy_evaluation(tinyw):
    vi = O.value_iteration(tinyw, tol=1e-12)
    V, Q = vi["V"], vi["Q"]
    n = tinyw.H * tinyw.W
    pi = Q.argmax(0)
    T = brute.dense_T(tinyw)
    R = brute.dense_R(tinyw, T)
    Tpi = T[pi, np.arange(n)]
    Rpi = R[pi, np.arange(n)]
    dead = tinyw.occ.ravel().astype(bool).copy()
    dead[tinyw.goal] = True
    Tpi[dead] = 0.0
    Rpi[dead] = 0.0
    Vpi = np.linalg.solve(np.eye(n) - tinyw.discount * Tpi, Rpi)
    g = tinyw.discount
    assert np.abs(Vpi - V).max() <= 1e-12 * g / (1 - g) * 10 + 1e-9


def test_vi_matches_dense_brute_force():
    for seed in range(3):
        w = WL.tiny(seed, H=8, W=7)
        vi = O.value_iteration(w, tol=1e-13)
        V, Q = brute.value_iteration(w, tol=1e-13)
        assert np.allclose(vi["V"], V, atol=1e-9)
        assert np.allclose(vi["Q"], Q, atol=1e-9)


def test_vi_truncated_runs_exact_sweeps():
    w = WL.diff(0, H=10, W=10)
    vi = O.value_iteration(w, truncated=37)
    assert vi["sweeps"] == 37 and len(vi["hist"]) == 37


def test_leaf_value_of_delta_is_state_value(tinyw):
    vi = O.value_iteration(tinyw, tol=1e-12)
    for s in np.flatnonzero(tinyw.occ.ravel() == 0)[:20]:
        b = np.zeros(tinyw.H * tinyw.W)
        b[s] = 1
        v, _ = O.leaf_value(tinyw, vi["Q"], b)
        if s == tinyw.goal:
            assert v == 0.0
        else:
            assert v == pytest.approx(vi["V"][s], abs=1e-10)


# ------------------------------------------------------------------ sampler
def test_sampler_frequencies_chi_square():
    P = np.array([0.05, 0.3, 0.15, 0.4, 0.1])
    N = 20000
    cnt = np.zeros(5)
    for k in range(N):
        cnt[O.sample_obs(P, O.uniform(77, 1, 0, 3, k))] += 1
    chi2 = ((cnt - N * P) ** 2 / (N * P)).sum()
    assert chi2 < 18.5          # 4 dof, p ~ 0.001


def test_sampler_inverts_cdf_at_known_points():
    P = np.array([0.25, 0.25, 0.5])
    assert O.sample_obs(P, 0.1) == 0
    assert O.sample_obs(P, 0.2499) == 0
    assert O.sample_obs(P, 0.25) == 1        # strict '<' against C(z)
    assert O.sample_obs(P, 0.49) == 1
    assert O.sample_obs(P, 0.5) == 2
    assert O.sample_obs(P, 0.9999) == 2
    assert O.is_boundary(P, 0.2500004) and O.is_boundary(P, 0.4999995)
    assert not O.is_boundary(P, 0.26) and not O.is_boundary(P, 0.9999995)


def test_ancestral_sampler_matches_marginal(tinyw):
    """Alg. 4 draws x ~ b, x' ~ T(x, a, .), z ~ O(x', .); its z has the law
    P(z | b, a) the oracle computes (Eq. 3 denominator)."""
    rng = np.random.default_rng(11)
    T = brute.dense_T(tinyw)
    Om = brute.dense_O(tinyw)
    b = _rand_belief(tinyw, 2)
    a = 1
    P = O.obs_marginal(tinyw, O.predict(tinyw, b, a))
    N = 40000
    x = rng.choice(len(b), size=N, p=b)
    cdfT = np.cumsum(T[a], axis=1)
    xp = (rng.random(N)[:, None] < cdfT[x]).argmax(1)
    cdfO = np.cumsum(Om, axis=1)
    z = (rng.random(N)[:, None] < cdfO[xp]).argmax(1)
    cnt = np.bincount(z, minlength=len(P))
    chi2 = ((cnt - N * P) ** 2 / (N * P)).sum()
    assert chi2 < 20.5          # 4 dof at B = 4, p ~ 0.0004


# ------------------------------------------------------------------ tree
def test_tree_depth0_is_qmdp(tinyw):
    vi = O.value_iteration(tinyw)
    tr = O.tree_plan(tinyw, vi["Q"], depth=0)
    v, qa = O.leaf_value(tinyw, vi["Q"], tinyw.b0)
    assert tr["root_value"] == pytest.approx(v, abs=1e-12)
    assert tr["root_action"] == int(np.argmax(qa))


def test_tree_marginal_with_full_coverage_equals_expectimax():
    # alpha = 0.6 and B = 1 make every observation likely, so K = 96 samples
    # cover both of them at every Q-node; MARGINAL weights are then P(z).
    for seed in range(3):
        w = WL.tiny(seed, H=5, W=6)
        w.beacons = w.beacons[:1]
        w.accuracy = 0.6
        vi = O.value_iteration(w, tol=1e-12)
        # normalise in FP64: MARGINAL weights renormalise over the sampled z,
        # expectimax does not, so b0 must sum to 1 beyond float32 rounding
        b0 = w.b0.astype(np.float64) / w.b0.astype(np.float64).sum()
        tr = O.tree_plan(w, vi["Q"], depth=2, K=96, weight_mode=O.MARGINAL, b0=b0)
        for l in range(2):
            cover = tr["n_level"][l + 1] == tr["n_level"][l] * 5 * (w.B + 1)
            assert cover, "K did not cover every observation"
        want = brute.expectimax(w, vi["Q"], b0, 2)
        assert tr["root_value"] == pytest.approx(want, abs=1e-10)


def test_tree_freq_converges_to_expectimax():
    w = WL.tiny(4, H=5, W=5)
    w.beacons = w.beacons[:2]
    vi = O.value_iteration(w, tol=1e-12)
    want = brute.expectimax(w, vi["Q"], w.b0, 1)
    vals = np.array([O.tree_plan(w, vi["Q"], depth=1, K=64, seed=s)["root_value"]
                     for s in range(40)])
    se = vals.std(ddof=1) / math.sqrt(len(vals)) + 1e-12
    assert abs(vals.mean() - want) < 4 * se + 1e-9


def test_tree_structure_invariants(tinyw):
    vi = O.value_iteration(tinyw)
    tr = O.tree_plan(tinyw, vi["Q"], depth=2, K=4, store_levels=2)
    lab = O.labels(tinyw)
    for l in range(1, 3):
        par, act, obs, wt = tr["parent"][l], tr["action"][l], tr["obs"][l], tr["weight"][l]
        key = par.astype(np.int64) * 1000 + act * 100 + obs
        assert (np.diff(key) > 0).all()          # (parent, action, z) ascending, unique
        for i in range(tr["n_level"][l - 1]):
            for a in range(5):
                m = (par == i) & (act == a)
                assert wt[m].sum() == pytest.approx(1.0, abs=1e-12)
                # the unique sampled z with their frequencies
                s = tr["samples"][l - 1][i, a]
                zs, cnt = np.unique(s, return_counts=True)
                assert list(obs[m]) == list(zs)
                assert np.allclose(wt[m], cnt / 4)
        B = tr["belief"][l]
        assert np.allclose(B.sum(1), 1.0, atol=1e-12)
        assert (B >= 0).all()
        # each child is Phi(parent, a, z)
        for j in range(0, tr["n_level"][l], 7):
            pb = tr["belief"][l - 1][par[j]]
            want, pz = O.correct(tinyw, O.predict(tinyw, pb, act[j]), obs[j], lab)
            assert np.allclose(B[j], want, atol=1e-15)
            assert tr["pz"][l][j] == pytest.approx(pz, abs=1e-15)


def test_tree_replay_reproduces_samples(tinyw):
    vi = O.value_iteration(tinyw)
    tr = O.tree_plan(tinyw, vi["Q"])
    tr2 = O.tree_plan(tinyw, vi["Q"], replay=tr["samples_flat"])
    assert tr2["root_value"] == tr["root_value"]
    assert np.array_equal(tr2["samples_flat"], tr["samples_flat"])


def test_tree_sample_stream_depends_on_path_only(tinyw):
    """The Philox counter names the (level, path) of a Q-node, so a node's
    samples do not depend on which other nodes were expanded."""
    vi = O.value_iteration(tinyw)
    tr = O.tree_plan(tinyw, vi["Q"], depth=2)
    nz = tinyw.B + 1
    for j in range(tr["n_level"][1]):
        a0, z0 = tr["action"][1][j], tr["obs"][1][j]
        for a in range(5):
            path = (a0 * nz + z0) * 5 + a
            us = [O.uniform(tinyw.seed, tinyw.episode, 1, path, k) for k in range(tinyw.K)]
            want = []
            P = O.obs_marginal(tinyw, O.predict(tinyw, tr_belief(tinyw, vi, tr, j), a))
            for u in us:
                want.append(O.sample_obs(P, u))
            assert list(tr["samples"][1][j, a]) == want


def tr_belief(w, vi, tr, j):
    full = O.tree_plan(w, vi["Q"], depth=2, store_levels=1)
    return full["belief"][1][j]
