"""Pins for the oracle's ancestral forward sampler (Alg. 4 as written):
its measurements follow the exact marginal P(z | b, a) = sum_x' O(x', z)
sum_x T(x, a, x') b(x) (Eq. 3's normaliser, from dense matrices), the law
the tree's inverse-CDF sampler draws from; from a one-cell belief every
sample reaches a successor of that cell.  None of these call the CUDA
library."""
import numpy as np
import pytest
from scipy.stats import chisquare

import oracle as O
from paper_1810_00204_gb300 import workloads as WL

import brute


@pytest.mark.parametrize("seed,a", [(0, 0), (1, 2), (2, 4)])
def test_ancestral_samples_follow_the_marginal(seed, a):
    w = WL.tiny(seed, H=10, W=11)
    rng = np.random.default_rng(seed)
    free = np.flatnonzero(w.occ.ravel() == 0)
    b = np.zeros(w.H * w.W)
    b[free] = rng.random(len(free))
    b /= b.sum()
    K = 20000
    z = O.forward_sample(w, b, a, K, seed=3, episode=seed, level=1, path=17)
    P = brute.dense_O(w).T @ (brute.dense_T(w)[a].T @ b)
    keep = P * K >= 5
    cnt = np.bincount(z, minlength=w.B + 1)
    fo = np.append(cnt[keep], cnt[~keep].sum())
    fe = np.append(P[keep], P[~keep].sum()) * K
    if fe[-1] == 0:
        fo, fe = fo[:-1], fe[:-1]
    assert chisquare(fo, fe).pvalue > 1e-4


def test_one_cell_belief_reaches_only_its_successors():
    w = WL.tiny(3, H=9, W=10)
    free = np.flatnonzero(w.occ.ravel() == 0)
    x = int(free[5]) if free[5] != w.goal else int(free[6])
    b = np.zeros(w.H * w.W)
    b[x] = 1.0
    T = brute.dense_T(w)
    lab = O.labels(w)
    for a in range(5):
        z = O.forward_sample(w, b, a, 4000, seed=5, level=2, path=a)
        # every measurement is possible at some successor, and the own labels
        # of the successors dominate (alpha = 0.9)
        succ = np.flatnonzero(T[a][x] > 0)
        own = set(int(lab[y]) for y in succ)
        frac = np.isin(z, list(own)).mean()
        assert frac > 0.85
