"""Dense numpy brute force of the paper's experimental model (Sec. V) on tiny
grids -- a second, independent formulation used to pin the model-9 oracle.
It builds T, R and O as dense matrices with vectorised shifts of the whole
grid (instead of per-cell transition rows), and evaluates the sampled tree
with dense matrix products.

The reading of the missing Fig. 2 is the oracle's: the stay action keeps the
robot in place; any other action reaches N_a(x) with probability 1 - 2 eps
and each of the two cells 45 degrees to either side with probability eps.
"""
import numpy as np

A, NZ = 9, 16
# action a -> (row step, col step) = (a // 3 - 1, a % 3 - 1)
STEP = {a: (a // 3 - 1, a % 3 - 1) for a in range(9)}
# the two 45-degree neighbours of each move direction (by angle, not index)
ANG = {a: np.arctan2(-(a // 3 - 1), a % 3 - 1) for a in range(9) if a != 4}


def _slips(a):
    """The two move directions 45 degrees from a's, found by angle."""
    out = []
    for b in ANG:
        d = np.angle(np.exp(1j * (ANG[b] - ANG[a])))
        if abs(abs(d) - np.pi / 4) < 1e-9:
            out.append(b)
    assert len(out) == 2
    return out


def _blocked(occ, d):
    """[H][W] bool: the cell at step d from each cell is occupied or outside."""
    H, W = occ.shape
    rr, cc = np.mgrid[0:H, 0:W]
    tr, tc = rr + d[0], cc + d[1]
    inside = (tr >= 0) & (tr < H) & (tc >= 0) & (tc < W)
    out = np.ones((H, W), bool)
    out[inside] = occ[tr[inside], tc[inside]] == 1
    return out


def _move(occ, d):
    """M[x, y] = 1 where the step d from x lands in y (blocked -> x)."""
    H, W = occ.shape
    n = H * W
    rr, cc = np.mgrid[0:H, 0:W]
    blk = _blocked(occ, d)
    dst = np.where(blk, rr * W + cc, (rr + d[0]) * W + (cc + d[1]))
    M = np.zeros((n, n))
    M[np.arange(n), dst.ravel()] = 1.0
    return M


def dense_T(w, slip=None):
    eps = w.slip if slip is None else slip
    occ = w.occ.astype(np.int64)
    n = w.H * w.W
    absorbing = occ.ravel() == 1
    absorbing[w.goal] = True
    T = np.zeros((A, n, n))
    for a in range(A):
        if a == 4:
            T[a] = np.eye(n)
            continue
        s1, s2 = _slips(a)
        T[a] = (1 - 2 * eps) * _move(occ, STEP[a]) + eps * _move(occ, STEP[s1]) + eps * _move(occ, STEP[s2])
        T[a][absorbing] = 0.0
        T[a][absorbing, absorbing.nonzero()[0]] = 1.0
    return T


def dense_R(w, slip=None):
    """R[a][x]: -2 for stay off the goal, else sum_y r(y) T'(x, a, y) with r
    = -2 on occupied (or outside) cells, 0 at the goal, -1 elsewhere; 0 at
    the goal and on occupied cells."""
    eps = w.slip if slip is None else slip
    occ = w.occ.astype(np.int64)
    H, W = occ.shape
    rr, cc = np.mgrid[0:H, 0:W]
    gr, gc = divmod(w.goal, W)

    def r_at(d):
        blk = _blocked(occ, d)
        at_goal = (rr + d[0] == gr) & (cc + d[1] == gc)
        return np.where(blk, -2.0, np.where(at_goal, 0.0, -1.0))

    R = np.zeros((A, H * W))
    for a in range(A):
        if a == 4:
            v = np.full((H, W), -2.0)
        else:
            s1, s2 = _slips(a)
            v = (1 - 2 * eps) * r_at(STEP[a]) + eps * r_at(STEP[s1]) + eps * r_at(STEP[s2])
        v = v.ravel().copy()
        v[occ.ravel() == 1] = 0.0
        v[w.goal] = 0.0
        R[a] = v
    return R


def dense_O(w, p_sensor=None):
    """O[x][z] = prod over the sensors (up, left, right, down = bits 0..3 of
    z) of p if the bit equals the cell's occupancy, else 1 - p."""
    ps = w.p_sensor if p_sensor is None else p_sensor
    occ = w.occ.astype(np.int64)
    bits = [_blocked(occ, d).ravel().astype(int) for d in ((-1, 0), (0, -1), (0, 1), (1, 0))]
    O = np.ones((w.H * w.W, NZ))
    for z in range(NZ):
        for j in range(4):
            O[:, z] *= np.where(bits[j] == (z >> j) & 1, ps, 1 - ps)
    return O


def value_iteration(w, sweeps=None, tol=1e-12, max_sweeps=100000):
    """Dense Jacobi value iteration; exactly `sweeps` sweeps when given."""
    T, R = dense_T(w), dense_R(w)
    V = np.zeros(w.H * w.W)
    k = 0
    while True:
        Vn = (R + w.discount * T @ V).max(axis=0)
        absorbing = w.occ.ravel() == 1
        absorbing[w.goal] = True
        Vn[absorbing] = 0.0
        res = np.abs(Vn - V).max()
        V = Vn
        k += 1
        if sweeps is not None:
            if k == sweeps:
                break
        elif res < tol or k >= max_sweeps:
            break
    Q = R + w.discount * T @ V
    return V, Q, k
