"""Dense numpy brute force for tiny grids -- a second, independent formulation
used to pin the oracle.  It builds every model matrix densely from the
problem statement (Sec. II, Eq. 10, the beacon sensor) with vectorised
shifts instead of per-cell transition rows, and evaluates the tree by full
expectimax over every observation (Eq. 2) instead of sampling.
"""
import numpy as np

A = 5
# action -> (row step, col step); perpendiculars of a move
STEP = {0: (-1, 0), 1: (0, 1), 2: (1, 0), 3: (0, -1)}
PERP = {0: (1, 3), 2: (1, 3), 1: (0, 2), 3: (0, 2)}


def _target_matrix(occ, d):
    """M[x, y] = 1 where moving from x by step d lands in y (blocked -> x)."""
    H, W = occ.shape
    n = H * W
    M = np.zeros((n, n))
    rr, cc = np.mgrid[0:H, 0:W]
    tr, tc = rr + d[0], cc + d[1]
    inside = (tr >= 0) & (tr < H) & (tc >= 0) & (tc < W)
    ok = inside.copy()
    ok[inside] &= occ[tr[inside], tc[inside]] == 0
    src = (rr * W + cc).ravel()
    dst = np.where(ok, tr * W + tc, rr * W + cc).ravel()
    M[src, dst] = 1.0
    return M


def dense_T(w, slip=None):
    """T[a] as dense n x n matrices, rows = from-state."""
    eps = w.slip if slip is None else slip
    occ = w.occ.astype(np.int64)
    n = w.H * w.W
    absorbing = (occ.ravel() == 1)
    absorbing[w.goal] = True
    T = np.zeros((A, n, n))
    for a in range(4):
        T[a] = (1 - 2 * eps) * _target_matrix(occ, STEP[a])
        for p in PERP[a]:
            T[a] += eps * _target_matrix(occ, STEP[p])
    T[4] = np.eye(n)
    for a in range(A):
        T[a][absorbing] = 0.0
        T[a][absorbing, absorbing.nonzero()[0]] = 1.0
    return T


def dense_labels(w):
    H, W = w.H, w.W
    rr, cc = np.mgrid[0:H, 0:W]
    best = np.full((H, W), w.B)
    bestd = np.full((H, W), np.inf)
    for k, bcell in enumerate(w.beacons):
        br, bc = divmod(int(bcell), W)
        d = np.abs(rr - br) + np.abs(cc - bc)
        take = (d <= w.sense_range) & (d < bestd)
        best[take] = k
        bestd[take] = d[take]
    return best.ravel()


def dense_O(w, accuracy=None):
    acc = w.accuracy if accuracy is None else accuracy
    lab = dense_labels(w)
    n, nz = w.H * w.W, w.B + 1
    O = np.full((n, nz), (1 - acc) / w.B)
    O[np.arange(n), lab] = acc
    return O


def dense_R(w, T=None, cost=None):
    T = dense_T(w) if T is None else T
    n = w.H * w.W
    c = np.zeros(n) if cost is None else np.asarray(cost, float).ravel()
    r = -1.0 - c
    r[w.goal] = 100.0
    R = np.einsum("axy,y->ax", T, r)
    dead = w.occ.ravel().astype(bool).copy()
    dead[w.goal] = True
    R[:, dead] = 0.0
    return R


def value_iteration(w, tol=1e-12, max_sweeps=100000):
    T = dense_T(w)
    R = dense_R(w, T, w.cost)
    dead = w.occ.ravel().astype(bool).copy()
    dead[w.goal] = True
    V = np.zeros(w.H * w.W)
    for _ in range(max_sweeps):
        Qs = R + w.discount * np.einsum("axy,y->ax", T, V)
        Vn = np.where(dead, 0.0, Qs.max(0))
        if np.abs(Vn - V).max() < tol:
            V = Vn
            break
        V = Vn
    Qs = R + w.discount * np.einsum("axy,y->ax", T, V)
    Qs[:, dead] = 0.0
    return V, Qs


def expectimax(w, Q, b, depth):
    """Full-width Eq. 2 recursion to depth d with QMDP leaves (Eq. 4)."""
    T = dense_T(w)
    O = dense_O(w)
    R = dense_R(w, T, w.cost)
    free = 1.0 - w.occ.ravel()

    def V(b, d):
        if d == 0:
            return float((Q @ b).max())
        best = -np.inf
        for a in range(A):
            bbar = T[a].T @ b
            q = float(R[a] @ b)
            for z in range(w.B + 1):
                pz = float(O[:, z] @ bbar)
                q += w.discount * pz * V(O[:, z] * bbar / pz, d - 1)
            best = max(best, q)
        return best

    return V(np.asarray(b, float).ravel() * free, depth)
