"""FP64 CPU oracle for QV-Tree Search -- test infrastructure only.

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg may import this package.  It wraps `qv_oracle.c` (plain C, FP64) through
ctypes and shares nothing with the CUDA library: its own build, its own
loader, its own unpadded [H][W] layout.  Inputs come from
`paper_1810_00204_gb300.workloads` (seeded generators, no method arithmetic).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qv_oracle.c")
_SRC9 = os.path.join(_HERE, "qv_oracle9.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

FREQ, MARGINAL = 0, 1
A = 5


def build(force: bool = False) -> str:
    """Compile qv_oracle.c into liboracle.so (gcc, OpenMP over tree nodes)."""
    srcs = [_SRC, _SRC9, os.path.join(_HERE, "qv_oracle.h"), os.path.join(_HERE, "qv_oracle9.h")]
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(map(os.path.getmtime, srcs)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC, _SRC9, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [("H", C.c_int), ("W", C.c_int), ("occ", C.c_void_p), ("B", C.c_int),
                ("beacon", C.c_void_p), ("range", C.c_int), ("goal", C.c_int),
                ("slip", C.c_double), ("acc", C.c_double), ("gamma", C.c_double),
                ("cost", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER(_Problem)
        vp = C.c_void_p
        L.or_labels.argtypes = [P, vp]
        L.or_transition_row.argtypes = [P, C.c_int, C.c_int, vp, vp]
        L.or_transition_row.restype = C.c_int
        L.or_reward_table.argtypes = [P, vp]
        L.or_value_iteration.argtypes = [P, C.c_double, C.c_int, C.c_int, vp, vp, vp, vp, vp]
        L.or_value_iteration.restype = C.c_int
        L.or_predict.argtypes = [P, vp, C.c_int, vp]
        L.or_obs_marginal.argtypes = [P, vp, vp, vp]
        L.or_correct.argtypes = [P, vp, vp, C.c_int, vp]
        L.or_correct.restype = C.c_double
        L.or_belief_reward.argtypes = [P, vp, vp, C.c_int]
        L.or_belief_reward.restype = C.c_double
        L.or_leaf_value.argtypes = [P, vp, vp, vp]
        L.or_leaf_value.restype = C.c_double
        L.or_philox4x32_10.argtypes = [vp, vp, vp]
        L.or_uniform.argtypes = [C.c_uint64, C.c_uint32, C.c_int, C.c_uint64, C.c_int]
        L.or_uniform.restype = C.c_float
        L.or_sample_obs.argtypes = [vp, C.c_int, C.c_float]
        L.or_sample_obs.restype = C.c_int
        L.or_is_boundary.argtypes = [vp, C.c_int, C.c_float]
        L.or_is_boundary.restype = C.c_int
        L.or_tree_plan.argtypes = [P, vp, vp, C.c_int, C.c_int, C.c_uint64, C.c_uint32, C.c_int,
                                   vp, vp, C.c_int] + [vp] * 16
        L.or_tree_plan.restype = C.c_int
        L.or_num_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        L.or_set_threads.restype = None
        L.or_transition_row_dslip.argtypes = [P, C.c_int, C.c_int, vp, vp]
        L.or_transition_row_dslip.restype = C.c_int
        L.or_tree_backward.argtypes = [P, vp, C.c_int, C.c_int, vp, vp, vp, vp, vp, vp, vp, vp,
                                       C.c_double, vp, vp, vp, vp, vp]
        L.or_tree_backward.restype = C.c_int
        L.or_vi_backward.argtypes = [P, C.c_int, vp, vp, vp, vp]
        L.or_vi_backward.restype = C.c_int
        L.or_fib_sweep.argtypes = [P, vp, vp, vp, vp]
        L.or_fib_sweep.restype = C.c_double
        L.or_fib_iteration.argtypes = [P, C.c_double, C.c_int, C.c_int, vp, vp, vp, vp]
        L.or_fib_iteration.restype = C.c_int
        L.or_pbvi_init.argtypes = [P, vp]
        L.or_pbvi_init.restype = None
        L.or_pbvi_expand.argtypes = [P, vp, C.c_int, C.c_int, C.c_uint64, vp, vp, vp, vp]
        L.or_pbvi_expand.restype = C.c_int
        L.or_pbvi_backup.argtypes = [P, vp, C.c_int, vp, C.c_int, vp, vp, vp, vp, vp, vp]
        L.or_pbvi_backup.restype = C.c_int
        L.or_tree_bounds.argtypes = [C.c_int] + [vp] * 9 + [C.c_double] + [vp] * 6
        L.or_tree_bounds.restype = C.c_int
        L.or_bestfirst.argtypes = ([P, vp, vp, C.c_int, vp, C.c_int, C.c_uint64, C.c_uint32, C.c_int, C.c_int,
                                    C.c_int, vp, vp] + [vp] * 19)
        L.or_bestfirst.restype = C.c_int
        L.or_env_step.argtypes = [P, vp, C.c_int, C.c_int, C.c_uint64, C.c_uint32, C.c_int, vp]
        L.or_env_step.restype = C.c_int
        L.or_closed_loop.argtypes = [P, vp, C.c_int, vp, vp, C.c_int, C.c_int, C.c_uint64, C.c_int] + [vp] * 8
        L.or_closed_loop.restype = C.c_int
        L.or_forward_sample.argtypes = [P, vp, C.c_int, C.c_int, C.c_uint64, C.c_uint32, C.c_int, C.c_uint64, vp, vp]
        L.or_forward_sample.restype = None
        P9 = C.POINTER(_Problem9)
        L.or9_tprime_row.argtypes = [P9, C.c_int, C.c_int, vp, vp, vp]
        L.or9_tprime_row.restype = C.c_int
        L.or9_transition_row.argtypes = [P9, C.c_int, C.c_int, vp, vp]
        L.or9_transition_row.restype = C.c_int
        L.or9_reward_table.argtypes = [P9, vp]
        L.or9_reward_table.restype = None
        L.or9_pattern.argtypes = [P9, C.c_int]
        L.or9_pattern.restype = C.c_int
        L.or9_obs_lik.argtypes = [P9, C.c_int, C.c_int]
        L.or9_obs_lik.restype = C.c_double
        L.or9_value_iteration.argtypes = [P9, C.c_double, C.c_int, C.c_int, vp, vp, vp, vp]
        L.or9_value_iteration.restype = C.c_int
        L.or9_predict.argtypes = [P9, vp, C.c_int, vp]
        L.or9_predict.restype = None
        L.or9_obs_marginal.argtypes = [P9, vp, vp]
        L.or9_obs_marginal.restype = None
        L.or9_correct.argtypes = [P9, vp, C.c_int, vp]
        L.or9_correct.restype = C.c_double
        L.or9_belief_reward.argtypes = [P9, vp, vp, C.c_int]
        L.or9_belief_reward.restype = C.c_double
        L.or9_leaf_value.argtypes = [P9, vp, vp, vp]
        L.or9_leaf_value.restype = C.c_double
        L.or9_tree_plan.argtypes = ([P9, vp, vp, C.c_int, C.c_int, C.c_uint64, C.c_uint32, vp, C.c_int]
                                    + [vp] * 15)
        L.or9_tree_plan.restype = C.c_int
        _lib = L
    return _lib


class _Problem9(C.Structure):
    _fields_ = [("H", C.c_int), ("W", C.c_int), ("occ", C.c_void_p), ("goal", C.c_int),
                ("slip", C.c_double), ("p_sensor", C.c_double), ("gamma", C.c_double)]


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


class Problem:
    """The model tuple of Sec. II built from a Workload (arrays kept alive)."""

    def __init__(self, w, slip=None, accuracy=None, cost="workload", discount=None):
        self.w = w
        self.H, self.W = w.H, w.W
        self.n = w.H * w.W
        self.B = w.B
        self.occ = np.ascontiguousarray(w.occ.reshape(-1), np.uint8)
        self.beacons = np.ascontiguousarray(w.beacons, np.int32)
        c = w.cost if isinstance(cost, str) else cost
        self.cost = None if c is None else np.ascontiguousarray(np.asarray(c, np.float64).reshape(-1))
        self.slip = w.slip if slip is None else slip
        self.acc = w.accuracy if accuracy is None else accuracy
        self.discount = w.discount if discount is None else discount
        self.s = _Problem(self.H, self.W, self.occ.ctypes.data, self.B, self.beacons.ctypes.data,
                          w.sense_range, w.goal, self.slip, self.acc, self.discount,
                          None if self.cost is None else self.cost.ctypes.data)
        self.ref = C.byref(self.s)


def _prob(w, **kw):
    return w if isinstance(w, Problem) else Problem(w, **kw)


def labels(w):
    p = _prob(w)
    out = np.zeros(p.n, np.int32)
    lib().or_labels(p.ref, _p(out))
    return out


def transition_row(w, x, a):
    p = _prob(w)
    y = np.zeros(4, np.int32)
    pr = np.zeros(4, np.float64)
    m = lib().or_transition_row(p.ref, int(x), int(a), _p(y), _p(pr))
    return {int(y[i]): float(pr[i]) for i in range(m)}


def reward_table(w):
    p = _prob(w)
    R = np.zeros(A * p.n, np.float64)
    lib().or_reward_table(p.ref, _p(R))
    return R.reshape(A, p.n)


def value_iteration(w, tol=None, max_sweeps=100000, truncated=None, **kw):
    """Returns dict(V [n], Q [5][n], sweeps, residual, hist, converged)."""
    p = _prob(w, **kw)
    ww = p.w
    tol = ww.vi_tol if tol is None else tol
    truncated = ww.vi_truncated if truncated is None else truncated
    V = np.zeros(p.n, np.float64)
    Q = np.zeros(A * p.n, np.float64)
    sw = C.c_int(0)
    res = C.c_double(0)
    hist = np.zeros(max(truncated, max_sweeps) + 1, np.float64)
    st = lib().or_value_iteration(p.ref, tol, max_sweeps, truncated, _p(V), _p(Q),
                                  C.byref(sw), C.byref(res), _p(hist))
    return dict(V=V, Q=Q.reshape(A, p.n), sweeps=sw.value, residual=res.value,
                hist=hist[:sw.value].copy(), converged=(st == 0))


def fib_iteration(w, tol=None, max_sweeps=100000, truncated=None, **kw):
    """Fast Informed Bound alpha-vectors (Sec. IV-A, Eq. 7) by Jacobi sweeps
    from alpha_0 = 0.  Returns dict(alpha [5][n], sweeps, residual, hist,
    converged).  V_FIB(b) (Eq. 6's value) is leaf_value(w, alpha, b)."""
    p = _prob(w, **kw)
    ww = p.w
    tol = ww.vi_tol if tol is None else tol
    truncated = ww.vi_truncated if truncated is None else truncated
    alpha = np.zeros(A * p.n, np.float64)
    sw = C.c_int(0)
    res = C.c_double(0)
    hist = np.zeros(max(truncated, max_sweeps) + 1, np.float64)
    st = lib().or_fib_iteration(p.ref, tol, max_sweeps, truncated, _p(alpha), C.byref(sw),
                                C.byref(res), _p(hist))
    return dict(alpha=alpha.reshape(A, p.n), sweeps=sw.value, residual=res.value,
                hist=hist[:sw.value].copy(), converged=(st == 0))


def fib_sweep(w, alpha, **kw):
    """One application of Eq. 7 to alpha [5][n]; returns (alpha', max change)."""
    p = _prob(w, **kw)
    label = labels(p)
    R = np.ascontiguousarray(reward_table(p).reshape(-1))
    a = np.ascontiguousarray(np.asarray(alpha, np.float64).reshape(-1))
    out = np.zeros(A * p.n, np.float64)
    res = lib().or_fib_sweep(p.ref, _p(label), _p(R), _p(a), _p(out))
    return out.reshape(A, p.n), res


def pbvi_init(w, **kw):
    """The pessimistic PBVI start alpha_0 [n] (R_min / (1 - gamma))."""
    p = _prob(w, **kw)
    out = np.zeros(p.n, np.float64)
    lib().or_pbvi_init(p.ref, _p(out))
    return out


def pbvi_expand(w, B, rnd, seed=None, **kw):
    """One round of belief set expansion (Sec. IV-B): a new point from each
    point of B [nB][n].  Returns dict(points [nB][n], action, obs, boundary)."""
    p = _prob(w, **kw)
    seed = p.w.seed if seed is None else seed
    B = np.ascontiguousarray(np.asarray(B, np.float64).reshape(-1, p.n))
    nB = B.shape[0]
    out = np.zeros_like(B)
    a = np.zeros(nB, np.int32)
    z = np.zeros(nB, np.int32)
    bd = np.zeros(nB, np.int32)
    lib().or_pbvi_expand(p.ref, _p(B), nB, int(rnd), int(seed), _p(out), _p(a), _p(z), _p(bd))
    return dict(points=out, action=a, obs=z, boundary=bd)


def pbvi_backup(w, B, G, want_score=False, **kw):
    """One Eq. 8 backup at every point of B [nB][n] given Gamma G [nG][n].
    Returns dict(G [nB][n], value, astar, best [nB][nz], q [nB][5], score
    [nB][5][nz][nG] or None)."""
    p = _prob(w, **kw)
    B = np.ascontiguousarray(np.asarray(B, np.float64).reshape(-1, p.n))
    G = np.ascontiguousarray(np.asarray(G, np.float64).reshape(-1, p.n))
    nB, nG, nz = B.shape[0], G.shape[0], p.B + 1
    Gout = np.zeros((nB, p.n), np.float64)
    value = np.zeros(nB, np.float64)
    astar = np.zeros(nB, np.int32)
    best = np.zeros((nB, nz), np.int32)
    q = np.zeros((nB, A), np.float64)
    score = np.zeros((nB, A, nz, nG), np.float64) if want_score else None
    lib().or_pbvi_backup(p.ref, _p(B), nB, _p(G), nG, _p(Gout), _p(value), _p(astar), _p(best), _p(q),
                         None if score is None else _p(score))
    return dict(G=Gout, value=value, astar=astar, best=best, q=q, score=score)


def pbvi_value(G, b):
    """V_PBVI(b) = max over the alpha-vectors of Gamma of alpha . b (Eq. 4's
    form with Gamma_PBVI); b [n] or [m][n]."""
    G = np.asarray(G, np.float64)
    return (np.asarray(b, np.float64) @ G.T).max(axis=-1)


def pbvi_solve(w, rounds, iters, seed=None, b0=None, **kw):
    """The PBVI schedule of this build: from B = {b0} and Gamma = {alpha_0},
    `rounds` times (`iters` backups of Eq. 8, then one expansion round),
    then `iters` more backups.  Returns dict(B, G, value, history)."""
    p = _prob(w, **kw)
    b = (p.w.b0.reshape(-1) if b0 is None else np.asarray(b0).reshape(-1)).astype(np.float64)
    B = b[None, :].copy()
    G = pbvi_init(p)[None, :]
    hist = []
    for r in range(rounds + 1):
        for _ in range(iters):
            bk = pbvi_backup(p, B, G)
            G = bk["G"]
            hist.append(bk["value"].copy())
        if r < rounds:
            B = np.concatenate([B, pbvi_expand(p, B, r, seed)["points"]])
    return dict(B=B, G=G, value=pbvi_value(G, B), history=hist)


def predict(w, b, a):
    p = _prob(w)
    b = np.ascontiguousarray(np.asarray(b, np.float64).reshape(-1))
    out = np.zeros(p.n, np.float64)
    lib().or_predict(p.ref, _p(b), int(a), _p(out))
    return out


def obs_marginal(w, bbar, label=None):
    p = _prob(w)
    label = labels(p) if label is None else label
    bbar = np.ascontiguousarray(np.asarray(bbar, np.float64).reshape(-1))
    P = np.zeros(p.B + 1, np.float64)
    lib().or_obs_marginal(p.ref, _p(label), _p(bbar), _p(P))
    return P


def correct(w, bbar, z, label=None):
    """Returns (b', P(z))."""
    p = _prob(w)
    label = labels(p) if label is None else label
    bbar = np.ascontiguousarray(np.asarray(bbar, np.float64).reshape(-1))
    out = np.zeros(p.n, np.float64)
    pz = lib().or_correct(p.ref, _p(label), _p(bbar), int(z), _p(out))
    return out, pz


def belief_reward(w, b, a, R=None):
    p = _prob(w)
    R = reward_table(p) if R is None else R
    R = np.ascontiguousarray(R, np.float64)
    b = np.ascontiguousarray(np.asarray(b, np.float64).reshape(-1))
    return lib().or_belief_reward(p.ref, _p(R), _p(b), int(a))


def leaf_value(w, Q, b):
    p = _prob(w)
    Q = np.ascontiguousarray(np.asarray(Q, np.float64).reshape(A, p.n))
    b = np.ascontiguousarray(np.asarray(b, np.float64).reshape(-1))
    qa = np.zeros(A, np.float64)
    v = lib().or_leaf_value(p.ref, _p(Q), _p(b), _p(qa))
    return v, qa


def philox(ctr, key):
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def uniform(seed, episode, level, path, k):
    return lib().or_uniform(seed, episode, level, path, k)


def sample_obs(P, u):
    P = np.ascontiguousarray(P, np.float64)
    return lib().or_sample_obs(_p(P), len(P), float(u))


def is_boundary(P, u):
    P = np.ascontiguousarray(P, np.float64)
    return bool(lib().or_is_boundary(_p(P), len(P), float(u)))


def level_capacity(B, K, depth):
    """Worst-case V-nodes per level: (5 * min(K, B+1))^l."""
    m = A * min(K, B + 1)
    return [m ** l for l in range(depth + 1)]


def tree_plan(w, Q, depth=None, K=None, seed=None, episode=None, weight_mode=FREQ,
              replay=None, store_levels=-1, b0=None, caps=None, **kw):
    """Level-synchronous QV-tree (Alg. 2-7).  Returns a dict with per-level
    arrays (lists indexed by level) and the root action / value / Q."""
    p = _prob(w, **kw)
    ww = p.w
    depth = ww.depth if depth is None else depth
    K = ww.K if K is None else K
    seed = ww.seed if seed is None else seed
    episode = ww.episode if episode is None else episode
    caps = level_capacity(p.B, K, depth) if caps is None else caps
    off = np.zeros(depth + 2, np.int64)
    off[1:] = np.cumsum(caps)
    tot = int(off[-1])
    Q = np.ascontiguousarray(np.asarray(Q, np.float64).reshape(A, p.n))
    b0 = ww.b0 if b0 is None else b0
    b0 = np.ascontiguousarray(np.asarray(b0, np.float64).reshape(-1))
    n_level = np.zeros(depth + 1, np.int32)
    parent = np.full(tot, -1, np.int32)
    action = np.full(tot, -1, np.int32)
    obs = np.full(tot, -1, np.int32)
    weight = np.zeros(tot, np.float64)
    pz = np.zeros(tot, np.float64)
    value = np.zeros(tot, np.float64)
    R = np.zeros(tot * A, np.float64)
    UQ = np.zeros(tot * A, np.float64)
    samples = np.full(tot * A * K, -1, np.int32)
    boundary = np.zeros(tot * A * K, np.uint8)
    belief = None
    if store_levels >= 0:
        nst = int(off[min(store_levels, depth) + 1])
        belief = np.zeros(nst * p.n, np.float64)
    if replay is not None:
        replay = np.ascontiguousarray(replay, np.int32)
    ra = C.c_int(0)
    rv = C.c_double(0)
    rq = np.zeros(A, np.float64)
    bc = C.c_long(0)
    st = lib().or_tree_plan(
        p.ref, _p(Q), _p(b0), depth, K, seed, episode, weight_mode,
        None if replay is None else _p(replay), _p(off), store_levels,
        _p(n_level), _p(parent), _p(action), _p(obs), _p(weight), _p(pz), _p(value),
        _p(R), _p(UQ), _p(samples), _p(boundary),
        None if belief is None else _p(belief), C.byref(ra), C.byref(rv), _p(rq), C.byref(bc))
    if st != 0:
        raise RuntimeError("oracle tree exceeded its level capacity")
    out = dict(root_action=ra.value, root_value=rv.value, root_q=rq, boundary_count=bc.value,
               n_level=n_level.copy(), off=off, depth=depth, K=K,
               samples_flat=samples, boundary_flat=boundary,
               flat=dict(n_level=n_level, parent=parent, action=action, obs=obs, weight=weight,
                         pz=pz, UQ=UQ, R=R, value=value, belief=belief, store_levels=store_levels))
    lv = {k: [] for k in ("parent", "action", "obs", "weight", "pz", "value", "R", "UQ",
                          "samples", "boundary", "belief")}
    for l in range(depth + 1):
        s, n = int(off[l]), int(n_level[l])
        lv["parent"].append(parent[s:s + n])
        lv["action"].append(action[s:s + n])
        lv["obs"].append(obs[s:s + n])
        lv["weight"].append(weight[s:s + n])
        lv["pz"].append(pz[s:s + n])
        lv["value"].append(value[s:s + n])
        lv["R"].append(R[s * A:(s + n) * A].reshape(n, A))
        lv["UQ"].append(UQ[s * A:(s + n) * A].reshape(n, A))
        lv["samples"].append(samples[s * A * K:(s + n) * A * K].reshape(n, A, K))
        lv["boundary"].append(boundary[s * A * K:(s + n) * A * K].reshape(n, A, K))
        if belief is not None and l <= store_levels:
            lv["belief"].append(belief[s * p.n:(s + n) * p.n].reshape(n, p.n))
    out.update(lv)
    return out


def tree_bounds(tree, Lleaf, gamma):
    """AEMS bookkeeping of Alg. 5-7 and Eq. 9 over a tree_plan tree given the
    lower bound of every leaf (Lleaf [n_leaves]).  Returns per-level lists
    LV, HV, EV (EV: index of a leaf in the deepest level) and LQ, HQ, EQ
    ([n][5], internal levels)."""
    f = tree["flat"]
    depth, off = tree["depth"], np.ascontiguousarray(tree["off"], np.int64)
    tot = int(off[-1])
    Ll = np.ascontiguousarray(np.asarray(Lleaf, np.float64).reshape(-1))
    assert Ll.size == int(f["n_level"][depth])
    LV = np.zeros(tot, np.float64)
    HV = np.zeros(tot, np.float64)
    EV = np.full(tot, -1, np.int32)
    LQ = np.zeros(tot * A, np.float64)
    HQ = np.zeros(tot * A, np.float64)
    EQ = np.full(tot * A, -1, np.int32)
    lib().or_tree_bounds(depth, _p(off), _p(f["n_level"]), _p(f["parent"]), _p(f["action"]), _p(f["weight"]),
                         _p(f["R"]), _p(f["UQ"]), _p(f["value"]), _p(Ll), float(gamma), _p(LV), _p(HV), _p(EV),
                         _p(LQ), _p(HQ), _p(EQ))
    out = {k: [] for k in ("LV", "HV", "EV", "LQ", "HQ", "EQ")}
    for l in range(depth + 1):
        s, n = int(off[l]), int(f["n_level"][l])
        out["LV"].append(LV[s:s + n])
        out["HV"].append(HV[s:s + n])
        out["EV"].append(EV[s:s + n])
        out["LQ"].append(LQ[s * A:(s + n) * A].reshape(n, A))
        out["HQ"].append(HQ[s * A:(s + n) * A].reshape(n, A))
        out["EQ"].append(EQ[s * A:(s + n) * A].reshape(n, A))
    return out


def bestfirst(w, Qu, G, iters, K=None, seed=None, episode=None, max_depth=6, max_nodes=None, b0=None, **kw):
    """Alg. 1's best-first planning loop: `iters` expansions of the V-node the
    root's E points at, U from the upper-bound alpha-vectors Qu [5][n] (FIB),
    L from the PBVI vectors G [nG][n].  Returns dict with per-node arrays
    (parent, action, obs, depth, weight, U, L, H, E, belief), per Q-node
    arrays [nodes][5] (R, UQ, LQ, HQ, EQ, first, count), expanded [iters],
    margin [iters] (the smallest gap among the comparisons that chose each
    iteration's node; inf while the root is a leaf), iterations, nodes,
    boundary, root_action."""
    p = _prob(w, **kw)
    ww = p.w
    K = ww.K if K is None else K
    seed = ww.seed if seed is None else seed
    episode = ww.episode if episode is None else episode
    nz = p.B + 1
    max_nodes = 1 + iters * A * min(K, nz) if max_nodes is None else max_nodes
    Qu = np.ascontiguousarray(np.asarray(Qu, np.float64).reshape(A, p.n))
    G = np.ascontiguousarray(np.asarray(G, np.float64).reshape(-1, p.n))
    b0 = ww.b0 if b0 is None else b0
    b0 = np.ascontiguousarray(np.asarray(b0, np.float64).reshape(-1))
    bel = np.zeros((max_nodes, p.n), np.float64)
    i32 = lambda m: np.zeros(m, np.int32)
    f64 = lambda m: np.zeros(m, np.float64)
    o = dict(expanded=i32(iters), parent=i32(max_nodes), action=i32(max_nodes), obs=i32(max_nodes),
             depth=i32(max_nodes), weight=f64(max_nodes), U=f64(max_nodes), L=f64(max_nodes), H=f64(max_nodes),
             E=i32(max_nodes), R=f64(max_nodes * A), UQ=f64(max_nodes * A), LQ=f64(max_nodes * A),
             HQ=f64(max_nodes * A), EQ=i32(max_nodes * A), first=i32(max_nodes * A), count=i32(max_nodes * A))
    nn = C.c_int(0)
    bd = C.c_long(0)
    margin = np.full(iters, np.inf, np.float64)
    it = lib().or_bestfirst(p.ref, _p(Qu), _p(G), G.shape[0], _p(b0), int(K), int(seed), int(episode), int(iters),
                            int(max_depth), int(max_nodes), _p(bel), C.byref(nn), _p(o["expanded"]),
                            _p(o["parent"]), _p(o["action"]), _p(o["obs"]), _p(o["depth"]), _p(o["weight"]),
                            _p(o["U"]), _p(o["L"]), _p(o["H"]), _p(o["E"]), _p(o["R"]), _p(o["UQ"]), _p(o["LQ"]),
                            _p(o["HQ"]), _p(o["EQ"]), _p(o["first"]), _p(o["count"]), C.byref(bd),
                            _p(margin))
    m = nn.value
    out = {k: v[:m] for k, v in o.items() if k != "expanded" and v.size == max_nodes}
    for k in ("R", "UQ", "LQ", "HQ", "EQ", "first", "count"):
        out[k] = o[k][:m * A].reshape(m, A)
    out["margin"] = margin
    out.update(expanded=o["expanded"], iterations=it, nodes=m, boundary=bd.value, belief=bel[:m],
               root_action=int(np.argmax(out["UQ"][0])) if out["count"][0].sum() else -1)
    return out


def env_step(w, x, a, seed, e, step):
    """The true system's step (motion outcome, then measurement): (x', z)."""
    p = _prob(w)
    z = C.c_int(0)
    y = lib().or_env_step(p.ref, _p(labels(p)), int(x), int(a), int(seed), int(e), int(step), C.byref(z))
    return y, z.value


def closed_loop(w, Q, b0s, x0s, depth=None, K=None, seed=None, max_steps=50, **kw):
    """E closed-loop episodes on the map of w (Alg. 1's outer loop): returns
    dict(actions, obs [E][S], states [E][S+1], steps, success, ret, root_gap
    [E][S], boundary [E][S])."""
    p = _prob(w, **kw)
    ww = p.w
    depth = ww.depth if depth is None else depth
    K = ww.K if K is None else K
    seed = ww.seed if seed is None else seed
    Q = np.ascontiguousarray(np.asarray(Q, np.float64).reshape(A, p.n))
    b0s = np.ascontiguousarray(np.asarray(b0s, np.float64).reshape(-1, p.n))
    x0s = np.ascontiguousarray(np.asarray(x0s, np.int32))
    E, S = b0s.shape[0], int(max_steps)
    o = dict(actions=np.zeros((E, S), np.int32), obs=np.zeros((E, S), np.int32),
             states=np.zeros((E, S + 1), np.int32), steps=np.zeros(E, np.int32), success=np.zeros(E, np.int32),
             ret=np.zeros(E, np.float64), root_gap=np.zeros((E, S), np.float64), boundary=np.zeros((E, S), np.int64))
    lib().or_closed_loop(p.ref, _p(Q), E, _p(b0s), _p(x0s), int(depth), int(K), int(seed), S, _p(o["actions"]),
                         _p(o["obs"]), _p(o["states"]), _p(o["steps"]), _p(o["success"]), _p(o["ret"]),
                         _p(o["root_gap"]), _p(o["boundary"]))
    return o


def forward_sample(w, b, a, K, seed=0, episode=0, level=0, path=0, want_boundary=False):
    """K measurements for (b, a) by Alg. 4's ancestral sampler: x ~ b,
    x' ~ T(x, a, .), z ~ O(x', .).  With want_boundary also the flags of
    draws whose x lies within 1e-5 of the total from a step of b's FP32
    cumulative sum."""
    p = _prob(w)
    b = np.ascontiguousarray(np.asarray(b, np.float64).reshape(-1))
    z = np.zeros(K, np.int32)
    bd = np.zeros(K, np.int32) if want_boundary else None
    lib().or_forward_sample(p.ref, _p(b), int(a), int(K), int(seed), int(episode), int(level), int(path), _p(z),
                            None if bd is None else _p(bd))
    return (z, bd) if want_boundary else z


def transition_row_dslip(w, x, a):
    """d T(x, a, y) / d eps for the targets y of row (x, a)."""
    p = _prob(w)
    y = np.zeros(4, np.int32)
    d = np.zeros(4, np.float64)
    m = lib().or_transition_row_dslip(p.ref, int(x), int(a), _p(y), _p(d))
    return {int(y[i]): float(d[i]) for i in range(m)}


def tree_backward(w, Q, tree, dL=1.0, **kw):
    """Adjoint of the root value of `tree` (a tree_plan result with
    store_levels >= depth - 1, FREQ weights).  Returns dict(Qbar [5][n],
    Rbar [5][n], dslip, dacc, db0 [n])."""
    p = _prob(w, **kw)
    f = tree["flat"]
    depth = tree["depth"]
    if f["belief"] is None or f["store_levels"] < max(depth - 1, 0):
        raise ValueError("tree_backward needs the beliefs of levels 0..depth-1")
    Q = np.ascontiguousarray(np.asarray(Q, np.float64).reshape(A, p.n))
    Qbar = np.zeros(A * p.n, np.float64)
    Rbar = np.zeros(A * p.n, np.float64)
    db0 = np.zeros(p.n, np.float64)
    ds = C.c_double(0.0)
    da = C.c_double(0.0)
    lib().or_tree_backward(p.ref, _p(Q), depth, tree["K"], _p(tree["off"]), _p(f["n_level"]),
                           _p(f["parent"]), _p(f["action"]), _p(f["obs"]), _p(f["weight"]),
                           _p(f["UQ"]), _p(f["belief"]), float(dL), _p(Qbar), _p(Rbar),
                           C.byref(ds), C.byref(da), _p(db0))
    return dict(Qbar=Qbar.reshape(A, p.n), Rbar=Rbar.reshape(A, p.n), dslip=ds.value,
                dacc=da.value, db0=db0)


def vi_backward(w, sweeps, Qbar, Rbar=None, **kw):
    """Adjoint of `sweeps` truncated VI sweeps and of R and Q.  Returns
    dict(dslip, dcost [n], Rbar [5][n] after the Q and sweep terms)."""
    p = _prob(w, **kw)
    Qbar = np.ascontiguousarray(np.asarray(Qbar, np.float64).reshape(-1))
    Rbar = np.zeros(A * p.n) if Rbar is None else np.array(Rbar, np.float64).reshape(-1)
    dcost = np.zeros(p.n, np.float64)
    ds = C.c_double(0.0)
    lib().or_vi_backward(p.ref, int(sweeps), _p(Qbar), _p(Rbar), C.byref(ds), _p(dcost))
    return dict(dslip=ds.value, dcost=dcost, Rbar=Rbar.reshape(A, p.n))


def root_value(w, sweeps, depth=None, K=None, seed=None, episode=None, replay=None, b0=None, **kw):
    """Root value of the plan on Q from `sweeps` truncated VI sweeps (FREQ
    weights; `replay` fixes the sampled measurements)."""
    p = _prob(w, **kw)
    vi = value_iteration(p, truncated=sweeps)
    t = tree_plan(p, vi["Q"], depth=depth, K=K, seed=seed, episode=episode, replay=replay, b0=b0)
    return t["root_value"], t


def root_value_grad(w, sweeps, depth=None, K=None, seed=None, episode=None, replay=None, b0=None,
                    dL=1.0, **kw):
    """Reverse mode of root_value: dict(value, dslip, dacc, dcost [n],
    db0 [n], tree)."""
    p = _prob(w, **kw)
    depth = p.w.depth if depth is None else depth
    vi = value_iteration(p, truncated=sweeps)
    t = tree_plan(p, vi["Q"], depth=depth, K=K, seed=seed, episode=episode, replay=replay, b0=b0,
                  store_levels=max(depth - 1, 0))
    tb = tree_backward(p, vi["Q"], t, dL=dL)
    vb = vi_backward(p, sweeps, tb["Qbar"], tb["Rbar"])
    return dict(value=t["root_value"], dslip=tb["dslip"] + vb["dslip"], dacc=tb["dacc"],
                dcost=vb["dcost"], db0=tb["db0"], tree=t, Q=vi["Q"])


def num_threads():
    return lib().or_num_threads()


def set_threads(n):
    """Threads of the oracle's parallel loops from now on."""
    lib().or_set_threads(int(n))


# ---------------------------------------------------------------------------
# The paper's experimental model (Sec. V): nine actions, four occupancy
# sensors (|Z| = 16), r in {-2, -1, 0}.  Thin wrappers over qv_oracle9.c.
A9, NZ9 = 9, 16


class Problem9:
    """The Sec. V model built from a Workload: its map, goal, slip (each
    45-degree slip), p_sensor and discount (arrays kept alive)."""

    def __init__(self, w, slip=None, p_sensor=None, discount=None):
        self.w = w
        self.H, self.W, self.n = w.H, w.W, w.H * w.W
        self.occ = np.ascontiguousarray(w.occ.reshape(-1).astype(np.uint8))
        self.s = _Problem9(self.H, self.W, self.occ.ctypes.data_as(C.c_void_p), int(w.goal),
                           float(w.slip if slip is None else slip),
                           float(w.p_sensor if p_sensor is None else p_sensor),
                           float(w.discount if discount is None else discount))
        self.ref = C.byref(self.s)


def _prob9(w, **kw):
    return w if isinstance(w, Problem9) else Problem9(w, **kw)


def tprime_row9(w, x, a, **kw):
    """T'(x, a, .) of the Fig. 2 reading: list of ((row, col), prob)."""
    p = _prob9(w, **kw)
    rr, cc, pr = (C.c_int * 3)(), (C.c_int * 3)(), (C.c_double * 3)()
    m = lib().or9_tprime_row(p.ref, int(x), int(a), rr, cc, pr)
    return [((rr[j], cc[j]), pr[j]) for j in range(m)]


def transition_row9(w, x, a, **kw):
    """Row x of T(x, a, .) of Sec. V: dict target -> probability."""
    p = _prob9(w, **kw)
    y, pr = (C.c_int * 3)(), (C.c_double * 3)()
    m = lib().or9_transition_row(p.ref, int(x), int(a), y, pr)
    return {y[j]: pr[j] for j in range(m)}


def reward_table9(w, **kw):
    p = _prob9(w, **kw)
    R = np.zeros(A9 * p.n)
    lib().or9_reward_table(p.ref, _p(R))
    return R.reshape(A9, p.n)


def pattern9(w, x, **kw):
    return lib().or9_pattern(_prob9(w, **kw).ref, int(x))


def obs_lik9(w, x, z, **kw):
    return lib().or9_obs_lik(_prob9(w, **kw).ref, int(x), int(z))


def value_iteration9(w, tol=None, max_sweeps=100000, truncated=0, **kw):
    """MDP value iteration on the Sec. V model: dict(V [n], Q [9][n], sweeps,
    residual, converged)."""
    p = _prob9(w, **kw)
    tol = p.w.vi_tol if tol is None else tol
    V = np.zeros(p.n)
    Q = np.zeros(A9 * p.n)
    sw = C.c_int(0)
    res = C.c_double(0.0)
    st = lib().or9_value_iteration(p.ref, float(tol), int(max_sweeps), int(truncated), _p(V), _p(Q),
                                   C.byref(sw), C.byref(res))
    return dict(V=V, Q=Q.reshape(A9, p.n), sweeps=sw.value, residual=res.value, converged=st == 0)


def predict9(w, b, a, **kw):
    p = _prob9(w, **kw)
    b = np.ascontiguousarray(np.asarray(b, np.float64).reshape(-1))
    out = np.zeros(p.n)
    lib().or9_predict(p.ref, _p(b), int(a), _p(out))
    return out


def obs_marginal9(w, bbar, **kw):
    p = _prob9(w, **kw)
    bbar = np.ascontiguousarray(np.asarray(bbar, np.float64).reshape(-1))
    P = np.zeros(NZ9)
    lib().or9_obs_marginal(p.ref, _p(bbar), _p(P))
    return P


def correct9(w, bbar, z, **kw):
    p = _prob9(w, **kw)
    bbar = np.ascontiguousarray(np.asarray(bbar, np.float64).reshape(-1))
    out = np.zeros(p.n)
    pz = lib().or9_correct(p.ref, _p(bbar), int(z), _p(out))
    return out, pz


def leaf_value9(w, Q, b, **kw):
    p = _prob9(w, **kw)
    Q = np.ascontiguousarray(np.asarray(Q, np.float64).reshape(-1))
    b = np.ascontiguousarray(np.asarray(b, np.float64).reshape(-1))
    qa = np.zeros(A9)
    v = lib().or9_leaf_value(p.ref, _p(Q), _p(b), _p(qa))
    return v, qa


def level_capacity9(K, depth):
    """Worst-case V-nodes per level of the nine-action tree."""
    caps = [1]
    for _ in range(depth):
        caps.append(caps[-1] * A9 * min(K, NZ9))
    return caps


def tree_plan9(w, Q, depth=None, K=None, seed=None, episode=None, b0=None, store_levels=-1, **kw):
    """The sampled tree (Alg. 2-7) on the Sec. V model; returns the node
    arrays of every level (flat, level l at off[l]) and the root."""
    p = _prob9(w, **kw)
    ww = p.w
    depth = ww.depth if depth is None else depth
    K = ww.K if K is None else K
    seed = ww.seed if seed is None else seed
    episode = ww.episode if episode is None else episode
    if depth > 3:
        raise ValueError("tree_plan9: depth <= 3")
    caps = level_capacity9(K, depth) + [0]
    off = np.zeros(depth + 3, np.int64)
    off[1:len(caps) + 1] = np.cumsum(caps)
    off[len(caps) + 1:] = off[len(caps)]
    total = int(off[depth + 1])
    Q = np.ascontiguousarray(np.asarray(Q, np.float64).reshape(-1))
    b = np.ascontiguousarray(np.asarray(ww.b0 if b0 is None else b0, np.float64).reshape(-1))
    n_level = np.zeros(depth + 1, np.int32)
    parent = np.full(total, -1, np.int32)
    action = np.full(total, -1, np.int32)
    obs = np.full(total, -1, np.int32)
    weight = np.zeros(total)
    pz = np.zeros(total)
    value = np.zeros(total)
    R = np.zeros(total * A9)
    UQ = np.zeros(total * A9)
    samples = np.full(total * A9 * K, -1, np.int32)
    boundary = np.zeros(total * A9 * K, np.uint8)
    nstore = int(off[min(store_levels, depth - 1) + 1]) if store_levels >= 0 and depth > 0 else 0
    belief = np.zeros(max(nstore, 1) * p.n) if nstore else None
    ra = C.c_int(0)
    rv = C.c_double(0.0)
    rq = np.zeros(A9)
    bc = C.c_long(0)
    st = lib().or9_tree_plan(p.ref, _p(Q), _p(b), int(depth), int(K), int(seed), int(episode), _p(off),
                             int(store_levels), _p(n_level), _p(parent), _p(action), _p(obs), _p(weight), _p(pz),
                             _p(value), _p(R), _p(UQ), _p(samples), _p(boundary),
                             _p(belief) if belief is not None else None, C.byref(ra), C.byref(rv), _p(rq),
                             C.byref(bc))
    if st != 0:
        raise RuntimeError("or9_tree_plan: capacity exceeded")
    return dict(n_level=n_level, off=off, parent=parent, action=action, obs=obs, weight=weight, pz=pz,
                value=value, R=R.reshape(-1, A9), UQ=UQ.reshape(-1, A9), samples=samples.reshape(-1, A9, K),
                boundary=boundary.reshape(-1, A9, K), belief=None if belief is None else belief.reshape(-1, p.n),
                root_action=ra.value, root_value=rv.value, root_q=rq, boundary_count=bc.value)
