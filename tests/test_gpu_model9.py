"""GPU parity of the paper's experimental model (Sec. V: nine actions, four
occupancy sensors) through the C ABI against the model-9 oracle: value
iteration sweep for sweep (FP64) and at convergence (FP32), whole trees on
small maps node by node, and at the mid map's planning configuration (d = 3,
K = 8) sampled nodes that the oracle recomputes one by one from the GPU's
own parent beliefs.  Tree shape, actions and measurements must match
exactly; values |d| <= 1e-5 * max(|ref|, 1) (FP32 against FP64, summed over
the whole tree: 1e-4)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1810_00204_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1810_00204_gb300 import api as A
    return A


def _close(got, ref, rel, what):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = max(1.0, float(np.abs(ref).max())) if ref.size else 1.0
    err = float(np.abs(got - ref).max()) if ref.size else 0.0
    assert err <= rel * scale, f"{what}: max |d| {err:.3e} > {rel:.1e} x {scale:.3g}"


@pytest.mark.parametrize("seed", [0, 4])
def test_value_iteration_fp64_sweeps(api, seed):
    w = WL.tiny(seed, H=17, W=23)
    m = api.Model9(w, depth=1, K=1)
    for k in (1, 9, 60):
        g = m.value_iterate("f64", truncated=k)
        o = O.value_iteration9(w, truncated=k)
        assert g["sweeps"] == k
        _close(g["V"].cpu().numpy().ravel(), o["V"], 1e-12, f"V after {k} sweeps")
        _close(g["Q"].cpu().numpy().reshape(9, -1), o["Q"], 1e-6, f"Q after {k} sweeps")


def test_value_iteration_fp32_converged(api):
    w = WL.mid(1, H=64, W=48)
    m = api.Model9(w, depth=1, K=1)
    g = m.value_iterate("f32", tol=1e-4)
    assert g["residual"] < 1e-4
    o = O.value_iteration9(w, truncated=g["sweeps"])
    _close(g["V"].cpu().numpy().ravel(), o["V"], 1e-5, "V")
    # the oracle stops at the same sweep within the FP32 residual's noise
    oc = O.value_iteration9(w, tol=1e-4)
    assert abs(oc["sweeps"] - g["sweeps"]) <= 2


def _compare_tree(api, w, depth, K):
    m = api.Model9(w, depth=depth, K=K)
    Qo = O.value_iteration9(w)["Q"]
    Qf = Qo.astype(np.float32)
    Q = torch.from_numpy(Qf.reshape(9, w.H, w.W)).cuda()
    g = m.plan(Q)
    o = O.tree_plan9(w, Qf.astype(np.float64), depth=depth, K=K, store_levels=depth - 1)
    assert o["boundary_count"] == 0, "pick a case without draws on a CDF step"
    assert g["nodes_per_level"] == [int(x) for x in o["n_level"]]
    for l in range(depth + 1):
        lv = m.level(l)
        n = lv["count"]
        s = slice(int(o["off"][l]), int(o["off"][l]) + n)
        assert np.array_equal(lv["parent"].cpu().numpy(), o["parent"][s]), l
        assert np.array_equal(lv["action"].cpu().numpy(), o["action"][s]), l
        assert np.array_equal(lv["obs"].cpu().numpy(), o["obs"][s]), l
        assert np.array_equal(lv["weight"].cpu().numpy(), o["weight"][s].astype(np.float32)), l
        _close(lv["pz"].cpu().numpy(), o["pz"][s], 1e-5, f"P(z) level {l}")
        _close(lv["value"].cpu().numpy(), o["value"][s], 1e-4, f"values level {l}")
        if l < depth:
            _close(lv["R"].cpu().numpy(), o["R"][s], 1e-5, f"R(b, a) level {l}")
            _close(lv["UQ"].cpu().numpy(), o["UQ"][s], 1e-4, f"U_Q level {l}")
            gb = lv["belief"].cpu().numpy().reshape(n, -1)
            ob = o["belief"][s]
            _close(gb, ob, 1e-5, f"beliefs level {l}")
    assert g["action"] == o["root_action"] or abs(o["root_q"][g["action"]] - o["root_value"]) <= 1e-4 * max(
        1.0, abs(o["root_value"]))
    _close([g["value"]], [o["root_value"]], 1e-5, "root value")


@pytest.mark.parametrize("seed,depth,K", [(0, 2, 4), (2, 2, 3), (1, 3, 2)])
def test_tree_matches_oracle(api, seed, depth, K):
    w = WL.tiny(seed, H=11, W=13)
    _compare_tree(api, w, depth, K)


def test_tree_with_obstacle_dense_map(api):
    w = WL.mid(3, H=24, W=20)
    _compare_tree(api, w, 2, 4)


def _oracle_path9(w, Qh, path):
    """The node reached from b0 along path [(a, z), ...], by the oracle: at
    every step its K draws on the marginal of its own belief must hold z.
    Returns (belief, P(z) of the last step, the draws' distinct z at the
    node for each action, lazily) or None when a draw on the way lies on a
    CDF step."""
    b = w.b0.ravel().astype(np.float64)
    code, pz = 0, None
    for l, (a, z) in enumerate(path):
        bbar = O.predict9(w, b, a)
        P = O.obs_marginal9(w, bbar)
        zs, bd = _draws9(w, P, l, code * 9 + a)
        if bd:
            return None
        assert z in zs, (l, a, z, zs)
        b, _ = O.correct9(w, bbar, z)
        pz = P[z]
        code = (code * 9 + a) * 16 + z
    return b, pz, code


def _draws9(w, P, level, path):
    zs, bd = [], False
    for k in range(w.K):
        u = O.lib().or_uniform(w.seed, w.episode, level, path, k)
        zs.append(O.lib().or_sample_obs(P.ctypes.data_as(O.C.c_void_p), 16, u))
        bd |= bool(O.lib().or_is_boundary(P.ctypes.data_as(O.C.c_void_p), 16, u))
    return sorted(set(zs)), bd


def test_full_size_sampled_nodes(api):
    # the mid map's planning configuration: 128 x 128, d = 3, K = 8, on the
    # oracle's Q.  The oracle's whole tree is too large here: sampled nodes
    # of the GPU's tree are recomputed by the oracle from b0 along their path
    # of (action, observation), each observation checked against the
    # oracle's own draws there
    w = WL.mid(0)
    m = api.Model9(w)
    Qo = O.value_iteration9(w, tol=1e-4)["Q"]
    Qf = Qo.astype(np.float32)
    g = m.plan(torch.from_numpy(Qf.reshape(9, w.H, w.W)).cuda())
    Qh = Qf.astype(np.float64)
    lv = [m.level(l) for l in range(4)]
    assert g["nodes_per_level"][0] == 1 and all(x > 0 for x in g["nodes_per_level"])
    # the backup identity at every internal node, in FP64 on the GPU's arrays
    for l in range(3):
        nxt = lv[l + 1]
        par, act = nxt["parent"].cpu().numpy(), nxt["action"].cpu().numpy()
        wv = (nxt["weight"].cpu().numpy().astype(np.float64) * nxt["value"].cpu().numpy())
        s = np.zeros((lv[l]["count"], 9))
        np.add.at(s, (par, act), wv)
        uq = lv[l]["R"].cpu().numpy() + w.discount * s
        _close(lv[l]["UQ"].cpu().numpy(), uq, 1e-5, f"U_Q identity level {l}")
        _close(lv[l]["value"].cpu().numpy(), uq.max(axis=1), 1e-5, f"U_V identity level {l}")
    arrays = [{k: lv[l][k].cpu().numpy() for k in ("parent", "action", "obs", "pz", "value")} for l in range(4)]

    def path_of(l, j):
        steps = []
        while l > 0:
            steps.append((int(arrays[l]["action"][j]), int(arrays[l]["obs"][j])))
            j = int(arrays[l]["parent"][j])
            l -= 1
        return list(reversed(steps))

    rng = np.random.default_rng(0)
    for l in (1, 2, 3):
        for j in rng.choice(lv[l]["count"], size=min(4, lv[l]["count"]), replace=False):
            got = _oracle_path9(w, Qh, path_of(l, int(j)))
            if got is None:
                continue
            bz, pz, code = got
            _close([float(arrays[l]["pz"][j])], [pz], 1e-5, f"P(z) of node {j} level {l}")
            if l < 3:
                _close(lv[l]["belief"][j].cpu().numpy().ravel(), bz, 1e-5, f"belief of node {j} level {l}")
                # the node's children for three actions: the oracle's draws
                for a in (0, 4, 7):
                    zs, bd = _draws9(w, O.obs_marginal9(w, O.predict9(w, bz, a)), l, code * 9 + a)
                    if bd:
                        continue
                    sel = (arrays[l + 1]["parent"] == j) & (arrays[l + 1]["action"] == a)
                    assert list(arrays[l + 1]["obs"][sel]) == zs, (l, int(j), a)
            else:
                v, _ = O.leaf_value9(w, Qh, bz)
                _close([float(arrays[l]["value"][j])], [v], 1e-5, f"leaf value of node {j}")
    _close([g["value"]], [lv[0]["value"][0].item()], 0.0, "root value read back")


def _edge(case):
    w = WL.tiny({"depth1": 0, "K16": 1, "exact": 2, "goal": 3}[case], H=11, W=13)
    depth, K = {"depth1": (1, 4), "K16": (2, 16), "exact": (2, 4), "goal": (2, 4)}[case]
    if case == "exact":
        w.slip, w.p_sensor = 0.0, 1.0
    if case == "goal":
        b = np.zeros((w.H, w.W), np.float32)
        b.ravel()[w.goal] = 1.0
        w.b0 = b
    return w, depth, K


@pytest.mark.parametrize("case", ["depth1", "K16", "exact", "goal"])
def test_tree_edge_cases(api, case):
    # the leaves one level below the root, the largest K, exact motion and
    # sensing, all of b0 on the (absorbing) goal
    w, depth, K = _edge(case)
    _compare_tree(api, w, depth, K)


def test_errors(api):
    import ctypes as C
    from paper_1810_00204_gb300 import _native as N
    w = WL.tiny(0, H=11, W=13)
    occ = torch.from_numpy(w.occ.astype(np.uint8)).cuda()

    def create(depth=2, K=4, slip=0.1, ps=0.95, goal=None):
        s = N.qv9_model_t(w.H, w.W, occ.data_ptr(), int(w.goal if goal is None else goal), slip, ps, 0.95)
        h = C.c_void_p()
        st = N.lib().qv9_create(C.byref(s), depth, K, C.byref(h))
        if st == 0:
            N.lib().qv9_destroy(h)
        return st

    assert create() == 0
    for kw in (dict(depth=0), dict(depth=4), dict(K=0), dict(K=17), dict(slip=0.5), dict(ps=0.4),
               dict(goal=int(np.flatnonzero(w.occ.ravel())[0]))):
        assert create(**kw) == N.QV_ERR_INVALID, kw
    m = api.Model9(w, depth=2, K=4)
    v = N.qv9_level_view_t()
    assert N.lib().qv9_level(m.handle, 0, C.byref(v)) == N.QV_ERR_INVALID  # no plan yet
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    p = small.data_ptr() + (-small.data_ptr()) % 256
    assert N.lib().qv9_set_workspace(m.handle, C.c_void_p(p), 256, None) == N.QV_ERR_WORKSPACE
