"""Pins for the oracle's reverse mode (the adjoint of the root value with
respect to the slip, the sensor accuracy, the cost map and b0): central finite
differences of the oracle's own forward pass with the sampled measurements
replayed, closed-form derivatives on a one-cell-wide corridor, and an
accuracy-independence invariant.  None of these call the CUDA library."""
import numpy as np
import pytest

import oracle as O
from paper_1810_00204_gb300 import workloads as WL

H_FD = 1e-6


def _problem(w, slip=None, acc=None, cost="workload", gamma=None):
    return O.Problem(w, slip=float(w.slip) if slip is None else slip,
                     accuracy=float(w.accuracy) if acc is None else acc,
                     cost=cost, discount=float(w.discount) if gamma is None else gamma)


def _small(seed=0, H=8, W=9, depth=2, K=4, cost=True):
    w = WL.tiny(seed, H=H, W=W, depth=depth, K=K)
    if cost:
        c = np.random.default_rng([7, seed]).uniform(0.0, 0.5, (H, W)).astype(np.float32)
        c.ravel()[w.goal] = 0.0
        w.cost = c
    return w


def _fd(f, x, h=H_FD):
    return (f(x + h) - f(x - h)) / (2 * h)


@pytest.mark.parametrize("seed,depth,K", [(0, 2, 4), (1, 3, 3), (2, 1, 8)])
def test_gradients_match_central_differences(seed, depth, K):
    w = _small(seed, depth=depth, K=K)
    S = 40
    cost = w.cost.astype(np.float64).ravel()
    b0 = w.b0.astype(np.float64).ravel()
    g = O.root_value_grad(_problem(w, cost=cost), S, depth=depth, K=K)
    rep = g["tree"]["samples_flat"]
    assert g["tree"]["boundary_count"] == 0

    def val(slip=None, acc=None, c=cost, b=b0):
        v, t = O.root_value(_problem(w, slip=slip, acc=acc, cost=c), S, depth=depth, K=K, replay=rep, b0=b)
        return v

    fd_slip = _fd(lambda s: val(slip=s), float(w.slip))
    fd_acc = _fd(lambda a: val(acc=a), float(w.accuracy))
    scale_s = max(1.0, abs(fd_slip))
    assert abs(g["dslip"] - fd_slip) < 1e-6 * scale_s
    assert abs(g["dacc"] - fd_acc) < 1e-6 * max(1.0, abs(fd_acc))
    # every cost cell
    fd_cost = np.zeros_like(cost)
    for i in range(cost.size):
        e = np.zeros_like(cost)
        e[i] = 1.0
        fd_cost[i] = _fd(lambda t: val(c=cost + t * e), 0.0)
    assert np.abs(g["dcost"] - fd_cost).max() < 1e-6 * max(1.0, np.abs(fd_cost).max())
    assert g["dcost"][w.goal] == 0.0
    assert np.all(g["dcost"][w.occ.ravel() == 1] == 0.0)
    # b0 on a few free cells, the largest adjoints first
    for i in np.argsort(-np.abs(g["db0"]))[:6]:
        e = np.zeros_like(b0)
        e[i] = 1.0
        fd = _fd(lambda t: val(b=b0 + t * e), 0.0)
        assert abs(g["db0"][i] - fd) < 1e-6 * max(1.0, abs(fd))


def _corridor(L, eps, gamma, cost=None, d=None):
    occ = np.zeros(L, np.uint8)
    b0 = np.zeros(L)
    b0[d] = 1.0
    w = WL.custom(1, L, occ, [0], 0, 0, d, eps, 0.9, gamma, b0, depth=0, K=1, cost=cost)
    return w


@pytest.mark.parametrize("eps,gamma", [(0.1, 0.95), (0.2, 0.9)])
def test_corridor_dslip_closed_form(eps, gamma):
    # Moving toward the goal on a one-cell-wide corridor, the perpendicular
    # slips are blocked: V(d) = N(d) / D with N = (1-2e)(r_{d-1} + g V(d-1)) - 2e,
    # D = 1 - 2 e g, so dV(d)/de = (N' + 2 g V(d)) / D with
    # N' = -2 (r_{d-1} + g V(d-1)) + (1-2e) g V'(d-1) - 2.
    L = 10
    V, dV = [0.0], [0.0]
    for d in range(1, L):
        r = 100.0 if d == 1 else -1.0
        N = (1 - 2 * eps) * (r + gamma * V[-1]) - 2 * eps
        D = 1 - 2 * eps * gamma
        Np = -2 * (r + gamma * V[-1]) + (1 - 2 * eps) * gamma * dV[-1] - 2
        V.append(N / D)
        dV.append((Np + 2 * gamma * V[-1]) / D)
    for d in (1, 2, 5, 9):
        w = _corridor(L, eps, gamma, d=d)
        g = O.root_value_grad(O.Problem(w, slip=eps, accuracy=0.9, cost=None, discount=gamma), 3000, depth=0, K=1)
        assert g["value"] == pytest.approx(V[d], abs=1e-9)
        assert g["dslip"] == pytest.approx(dV[d], rel=1e-9, abs=1e-9)


def test_corridor_dcost_closed_form():
    # eps = 0: V(d) = sum_{j=1..d} g^{j-1} r(d-j), r(0) = 100, r(y) = -1 - c(y),
    # so dV(d)/dc(d-j) = -g^{j-1} for j = 1..d-1 and 0 for every other cell.
    L, gamma = 9, 0.95
    c = np.random.default_rng(3).uniform(0.0, 0.5, L)
    c[0] = 0.0
    for d in (1, 4, 8):
        w = _corridor(L, 0.0, gamma, cost=c, d=d)
        g = O.root_value_grad(O.Problem(w, slip=0.0, accuracy=0.9, cost=c, discount=gamma), 200, depth=0, K=1)
        want = np.zeros(L)
        for j in range(1, d):
            want[d - j] = -gamma ** (j - 1)
        assert np.allclose(g["dcost"], want, atol=1e-12)
        assert g["dslip"] != 0.0 or d == 1


def test_accuracy_has_no_effect_when_every_cell_shares_a_label():
    # One beacon whose range covers the whole grid: O(., z) is constant over
    # the cells for every z, so every correction returns the predicted belief
    # and the FREQ-weighted root value does not depend on alpha.
    w = WL.tiny(4, H=6, W=6, depth=2, K=4)
    w.beacons = w.beacons[:1]
    w.sense_range = 20
    g = O.root_value_grad(_problem(w, cost=None), 30, depth=2, K=4)
    assert abs(g["dacc"]) < 1e-12 * max(1.0, abs(g["value"]))
    assert abs(g["dslip"]) > 1e-6


def test_gradient_is_linear_in_the_seed_adjoint():
    w = _small(5, depth=2, K=3)
    p = _problem(w, cost=w.cost.astype(np.float64).ravel())
    g1 = O.root_value_grad(p, 25, depth=2, K=3, dL=1.0)
    g2 = O.root_value_grad(p, 25, depth=2, K=3, dL=-2.5)
    assert g2["dslip"] == pytest.approx(-2.5 * g1["dslip"], rel=1e-12)
    assert g2["dacc"] == pytest.approx(-2.5 * g1["dacc"], rel=1e-12)
    assert np.allclose(g2["dcost"], -2.5 * g1["dcost"], rtol=1e-12, atol=1e-15)


def test_transition_dslip_is_derivative_of_row():
    w = _small(6)
    for x in range(w.H * w.W):
        for a in range(5):
            r0 = O.transition_row(_problem(w, slip=0.1), x, a)
            r1 = O.transition_row(_problem(w, slip=0.1 + 1e-3), x, a)
            d = O.transition_row_dslip(_problem(w, slip=0.1), x, a)
            for y in set(r0) | set(r1):
                fd = (r1.get(y, 0.0) - r0.get(y, 0.0)) / 1e-3
                assert d.get(y, 0.0) == pytest.approx(fd, abs=1e-9)
