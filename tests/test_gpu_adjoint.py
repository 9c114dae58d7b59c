"""Parity of the CUDA adjoint (mdp_value_iterate_checkpointed,
mdp_value_backward, qv_tree_backward and the torch.autograd.Function over
them) with the FP64 oracle's reverse mode, and with central finite
differences of the oracle's forward pass.

Tolerances: the value iteration and its adjoint run in FP64 on both sides
(different summation order only), so 1e-9 relative.  The tree's forward pass
is FP32 on the GPU (beliefs, P(z), values) and FP64 in the oracle; its
adjoint sums O(1e4) terms per node, so every gradient is held to the 1e-4
relative bound (norm-wise: max |gpu - ref| <= 1e-4 max |ref| for maps)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1810_00204_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

GRAD_REL = 1e-4
VI_REL = 1e-9
# Absolute floor for a scalar gradient whose exact value is (near) zero, for
# example d/d alpha when every active belief lies inside one label region:
# FP32 rounding of the forward beliefs (2^-24 relative) times adjoint terms of
# magnitude O(1e2) summed over the nodes leaves residues near 1e-6.
GRAD_ABS = 1e-5


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_1810_00204_gb300 import api as A
    return A


def _close(got, ref, rel, floor=1e-12, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = max(np.abs(ref).max(initial=0.0), floor)
    err = np.abs(got - ref).max(initial=0.0)
    assert err <= rel * scale, f"{what}: max err {err:.3e} > {rel:.0e} * {scale:.3e}"


def _with_cost(w, seed):
    c = np.random.default_rng([11, seed]).uniform(0.0, 0.5, (w.H, w.W)).astype(np.float32)
    c.ravel()[w.goal] = 0.0
    w.cost = c
    return w


def _spread(w):
    """b0 uniform over every free cell, so the active beliefs straddle label
    regions and the accuracy enters the root value."""
    free = (w.occ == 0).astype(np.float32)
    w.b0 = free / free.sum()
    return w


def _prob(w):
    return O.Problem(w, slip=float(w.slip), accuracy=float(w.accuracy), discount=float(w.discount),
                     cost=None if w.cost is None else w.cost.astype(np.float64).ravel())


def _tree_case(api, w, depth, K, sweeps, leaf_mode, every=16):
    """GPU VI (checkpointed) and plan on the GPU's Q; the oracle tree on the
    oracle's own Q of the same truncated VI, with its own samples, replayed
    into the GPU plan so both trees are the same."""
    m = api.Model(w)
    vi = api.mdp_value_iterate_checkpointed(m, sweeps, every)
    p = _prob(w)
    Qf = O.value_iteration(p, truncated=sweeps)["Q"]
    _close(m.from_grid(vi["Q"]).reshape(5, -1), Qf, 1e-6, floor=1.0, what="Q of the truncated VI")
    o = O.tree_plan(p, Qf, depth=depth, K=K, store_levels=max(depth - 1, 0))
    rep = torch.from_numpy(o["samples_flat"].copy()).cuda()
    r, plan = api.qv_tree_plan(m, vi["Q"], m.b0(), depth=depth, K=K, seed=w.seed, episode=w.episode,
                               leaf_mode=leaf_mode, replay=rep, keep=True)
    assert r["nodes_per_level"] == [int(x) for x in o["n_level"]]
    return m, vi, p, Qf, o, r, plan


# ------------------------------------------------------------------ value iteration
@pytest.mark.parametrize("make", [lambda: _with_cost(WL.tiny(0), 0), lambda: WL.tiny(3, H=17, W=23),
                                  lambda: WL.diff(0)])
def test_checkpointed_vi_matches_oracle_sweeps(api, make):
    w = make()
    S, c = 40, 16
    m = api.Model(w)
    vi = api.mdp_value_iterate_checkpointed(m, S, c)
    p = _prob(w)
    for j in range(vi["ckpt"].shape[0]):
        ref = O.value_iteration(p, truncated=j * c)["V"] if j > 0 else np.zeros(w.H * w.W)
        _close(m.from_grid(vi["ckpt"][j]), ref, VI_REL, floor=1.0, what=f"checkpoint {j}")
    o = O.value_iteration(p, truncated=S)
    _close(m.from_grid(vi["V"]), o["V"], VI_REL, floor=1.0, what="V_S")
    _close(m.from_grid(vi["Q"]).reshape(5, -1), o["Q"], 1e-6, floor=1.0, what="Q")


@pytest.mark.parametrize("make,S,every", [(lambda: _with_cost(WL.tiny(0), 0), 40, 16),
                                          (lambda: _with_cost(WL.tiny(1, H=13, W=31), 1), 33, 5),
                                          (lambda: WL.tiny(2), 17, 32),
                                          (lambda: WL.diff(0), 200, 16)])
def test_vi_backward_matches_oracle(api, make, S, every):
    """Without a cost map every action of an open cell earns -1 in the first
    sweeps, so the Bellman max is an exact tie whose pick depends on rounding:
    d/dc is then not unique (a kink at c = 0) and only d/d slip, which is the
    same for every tied action, is compared."""
    w = make()
    m = api.Model(w)
    vi = api.mdp_value_iterate_checkpointed(m, S, every)
    rng = np.random.default_rng(5)
    Qbar = rng.standard_normal((5, w.H * w.W))  # also on walls and the goal, which both sides ignore
    dslip = torch.zeros(1, dtype=torch.float64, device="cuda")
    dcost = torch.zeros((w.H, m.P), dtype=torch.float64, device="cuda")
    Qg = torch.zeros((5, w.H, m.P), dtype=torch.float64, device="cuda")
    Qg[:, :, :w.W] = torch.from_numpy(Qbar.reshape(5, w.H, w.W)).cuda()
    api.mdp_value_backward(m, vi, Qg, dslip, dcost)
    ref = O.vi_backward(_prob(w), S, Qbar)
    assert float(dslip[0]) == pytest.approx(ref["dslip"], rel=VI_REL, abs=1e-9)
    if w.cost is not None:
        _close(dcost[:, :w.W].cpu().numpy().ravel(), ref["dcost"], VI_REL, floor=1.0, what="dcost")


# ------------------------------------------------------------------ tree adjoint
@pytest.mark.parametrize("seed,depth,K,leaf_mode,spread", [(0, 2, 4, 0, False), (0, 2, 4, 1, False),
                                                           (1, 3, 3, 0, False), (1, 3, 3, 1, True),
                                                           (2, 1, 8, 0, True), (3, 2, 8, 0, False),
                                                           (4, 0, 4, 0, False), (5, 2, 6, 0, True),
                                                           (7, 3, 4, 1, True)])
def test_tree_backward_matches_oracle(api, seed, depth, K, leaf_mode, spread):
    w = _with_cost(WL.tiny(seed), seed)
    if spread:
        w = _spread(w)
    m, vi, p, Qf, o, r, plan = _tree_case(api, w, depth, K, 30, leaf_mode)
    tb = api.qv_tree_backward(plan, 0, dL=1.0)
    ob = O.tree_backward(p, Qf, o)
    conv = O.vi_backward(p, 0, np.zeros((5, w.H * w.W)), ob["Rbar"])  # R(b, a) into slip and cost
    torch.cuda.synchronize()
    _close(m.from_grid(tb["Qbar"]).reshape(5, -1), ob["Qbar"], GRAD_REL, floor=1e-6, what="Qbar")
    assert float(tb["dslip"][0]) == pytest.approx(ob["dslip"] + conv["dslip"], rel=GRAD_REL, abs=GRAD_ABS)
    assert float(tb["dacc"][0]) == pytest.approx(ob["dacc"], rel=GRAD_REL, abs=GRAD_ABS)
    if spread and depth > 0:
        assert abs(ob["dacc"]) > 1e3 * GRAD_ABS  # the accuracy does enter this tree
    _close(m.from_grid(tb["dcost"]), conv["dcost"], GRAD_REL, floor=1e-6, what="dcost")
    _close(m.from_grid(tb["db0"]), ob["db0"], GRAD_REL, floor=1e-6, what="db0")


def test_tree_backward_accumulates_and_repeats(api):
    w = _with_cost(WL.tiny(5), 5)
    m, vi, p, Qf, o, r, plan = _tree_case(api, w, 2, 4, 30, 0)
    a = api.qv_tree_backward(plan, 0, dL=1.0)
    b = api.qv_tree_backward(plan, 0, dL=1.0)
    for k in ("Qbar", "dslip", "dacc", "dcost", "db0"):
        _close(b[k].cpu().numpy(), a[k].cpu().numpy(), 1e-12, floor=1e-12, what=k)
    # accumulation into the same buffers, with a scaled seed adjoint
    api.qv_tree_backward(plan, 0, dL=-2.0, Qbar=a["Qbar"], dslip=a["dslip"], dacc=a["dacc"], dcost=a["dcost"],
                         db0=a["db0"])
    for k in ("Qbar", "dslip", "dacc", "dcost", "db0"):
        _close(a[k].cpu().numpy(), -b[k].cpu().numpy(), 1e-12, floor=1e-12, what=k + " accumulated")


def test_tree_backward_refuses_marginal_weights(api):
    from paper_1810_00204_gb300 import _native as N
    w = WL.tiny(0)
    m = api.Model(w)
    vi = api.mdp_value_iterate_checkpointed(m, 20, 16)
    r, plan = api.qv_tree_plan(m, vi["Q"], m.b0(), depth=2, K=4, weight_mode=N.QV_WEIGHT_MARGINAL, keep=True)
    with pytest.raises(N.QVError) as ei:
        api.qv_tree_backward(plan, 0)
    assert ei.value.status == N.QV_ERR_INVALID


# ------------------------------------------------------------------ end to end
def _full_grad_gpu(api, m, vi, plan):
    tb = api.qv_tree_backward(plan, 0, dL=1.0)
    api.mdp_value_backward(m, vi, tb["Qbar"], tb["dslip"], tb["dcost"])
    return (float(tb["dslip"][0]), float(tb["dacc"][0]), m.from_grid(tb["dcost"]), m.from_grid(tb["db0"]))


@pytest.mark.parametrize("seed,depth,K,leaf_mode", [(0, 2, 4, 0), (6, 3, 4, 1)])
def test_gradient_matches_oracle_and_finite_differences(api, seed, depth, K, leaf_mode):
    w = _spread(_with_cost(WL.tiny(seed), seed))
    S = 60
    m, vi, p, Qf, o, r, plan = _tree_case(api, w, depth, K, S, leaf_mode)
    ds, da, dc, db = _full_grad_gpu(api, m, vi, plan)
    rep = o["samples_flat"]
    ref = O.root_value_grad(p, S, depth=depth, K=K, replay=rep)
    assert ds == pytest.approx(ref["dslip"], rel=GRAD_REL)
    assert da == pytest.approx(ref["dacc"], rel=GRAD_REL, abs=GRAD_ABS)
    assert abs(ref["dacc"]) > 1e3 * GRAD_ABS
    _close(dc, ref["dcost"], GRAD_REL, what="dcost")
    _close(db, ref["db0"], GRAD_REL, what="db0")
    cost = w.cost.astype(np.float64).ravel()

    def val(slip=float(w.slip), acc=float(w.accuracy), c=cost):
        q = O.Problem(w, slip=slip, accuracy=acc, discount=float(w.discount), cost=c)
        return O.root_value(q, S, depth=depth, K=K, replay=rep)[0]

    h = 1e-6
    fd = (val(slip=float(w.slip) + h) - val(slip=float(w.slip) - h)) / (2 * h)
    assert ds == pytest.approx(fd, rel=GRAD_REL)
    fd = (val(acc=float(w.accuracy) + h) - val(acc=float(w.accuracy) - h)) / (2 * h)
    assert da == pytest.approx(fd, rel=GRAD_REL, abs=GRAD_ABS)
    for i in np.argsort(-np.abs(ref["dcost"]))[:3]:
        e = np.zeros_like(cost)
        e[i] = h
        fd = (val(c=cost + e) - val(c=cost - e)) / (2 * h)
        assert dc[i] == pytest.approx(fd, rel=GRAD_REL, abs=1e-8)


def test_autograd_function_on_the_differentiation_workload(api):
    """128x128, depth 3, K = 8, 200 truncated sweeps with checkpoints every
    16, a U[0, 0.5] cost map: torch.autograd through QVRootValue against the
    oracle's reverse mode and central differences of the oracle for the slip
    and the accuracy.  The oracle draws its own samples; the GPU's own draws
    are checked against them (identical away from flagged CDF steps), and the
    autograd plan replays the oracle's samples so both differentiate the same
    tree."""
    from paper_1810_00204_gb300.autograd import root_value
    w = WL.diff(0)
    p = _prob(w)
    own = O.tree_plan(p, O.value_iteration(p, truncated=200)["Q"], depth=3, K=8, seed=w.seed, episode=w.episode)
    rep = own["samples_flat"]
    # the GPU's own samples are the oracle's Philox draws (the samples depend
    # on the beliefs only, not on Q), except at draws the oracle flags as
    # lying within 1e-6 of a CDF step
    m = api.Model(w)
    vi = api.mdp_value_iterate_checkpointed(m, 200, 16)
    r, plan = api.qv_tree_plan(m, vi["Q"], m.b0(), depth=3, K=8, seed=w.seed, episode=w.episode, keep=True)
    assert own["n_level"].tolist() == r["nodes_per_level"] or own["boundary_count"] > 0
    for l in range(3):
        if plan.level(0, l)["count"] != own["n_level"][l]:
            break
        gs = plan.level(0, l)["samples"].cpu().numpy()
        assert not ((gs != own["samples"][l]) & (own["boundary"][l] == 0)).any(), f"level {l} samples"
    slip = torch.tensor(float(w.slip), dtype=torch.float64, requires_grad=True)
    acc = torch.tensor(float(w.accuracy), dtype=torch.float64, requires_grad=True)
    cost = torch.from_numpy(w.cost.copy()).cuda().requires_grad_(True)
    v = root_value(w, slip, acc, cost, depth=3, K=8, seed=w.seed, episode=w.episode, sweeps=200, every=16,
                   replay=torch.from_numpy(rep.copy()).cuda())
    v.backward()
    ref = O.root_value_grad(p, 200, depth=3, K=8, replay=rep)
    assert float(v.detach()) == pytest.approx(ref["value"], rel=1e-5)
    assert float(slip.grad) == pytest.approx(ref["dslip"], rel=GRAD_REL)
    assert float(acc.grad) == pytest.approx(ref["dacc"], rel=GRAD_REL, abs=GRAD_ABS)
    _close(cost.grad.cpu().numpy().ravel(), ref["dcost"], GRAD_REL, what="dcost")
    c64 = w.cost.astype(np.float64).ravel()

    def val(slip_v=float(w.slip), acc_v=float(w.accuracy)):
        q = O.Problem(w, slip=slip_v, accuracy=acc_v, discount=float(w.discount), cost=c64)
        return O.root_value(q, 200, depth=3, K=8, replay=rep)[0]

    h = 1e-6
    fd = (val(slip_v=float(w.slip) + h) - val(slip_v=float(w.slip) - h)) / (2 * h)
    assert float(slip.grad) == pytest.approx(fd, rel=GRAD_REL)
    fd = (val(acc_v=float(w.accuracy) + h) - val(acc_v=float(w.accuracy) - h)) / (2 * h)
    assert float(acc.grad) == pytest.approx(fd, rel=GRAD_REL, abs=GRAD_ABS)


def test_gradient_on_the_differentiation_workload_with_a_spread_belief(api):
    """The differentiation workload (128x128, depth 3, K = 8, 200 truncated
    sweeps with checkpoints every 16, its cost map) with b0 spread over every
    free cell, so that the active beliefs straddle label regions and
    d/d accuracy is far from zero (about 2e-2, two thousand times the
    absolute floor): the GPU's gradient against the oracle's reverse mode and
    central differences (h = 1e-6) at 1e-4 relative.  d/d accuracy is a
    difference of adjoint terms of order 1e2 whose forward inputs (P(z), leaf
    values) are FP32, so it keeps the 1e-5 absolute floor of the other
    scalar checks (a few 1e-6 of rounding are expected here)."""
    w = _spread(WL.diff(0))
    S = 200
    m, vi, p, Qf, o, r, plan = _tree_case(api, w, 3, 8, S, 0)
    ds, da, dc, db = _full_grad_gpu(api, m, vi, plan)
    rep = o["samples_flat"]
    ref = O.root_value_grad(p, S, depth=3, K=8, replay=rep)
    assert abs(ref["dacc"]) > 1e3 * GRAD_ABS
    assert ds == pytest.approx(ref["dslip"], rel=GRAD_REL)
    assert da == pytest.approx(ref["dacc"], rel=GRAD_REL, abs=GRAD_ABS)
    _close(dc, ref["dcost"], GRAD_REL, what="dcost")
    _close(db, ref["db0"], GRAD_REL, what="db0")
    cost = w.cost.astype(np.float64).ravel()

    def val(slip=float(w.slip), acc=float(w.accuracy), c=cost):
        q = O.Problem(w, slip=slip, accuracy=acc, discount=float(w.discount), cost=c)
        return O.root_value(q, S, depth=3, K=8, replay=rep)[0]

    h = 1e-6
    fd = (val(slip=float(w.slip) + h) - val(slip=float(w.slip) - h)) / (2 * h)
    assert ds == pytest.approx(fd, rel=GRAD_REL)
    fd = (val(acc=float(w.accuracy) + h) - val(acc=float(w.accuracy) - h)) / (2 * h)
    assert da == pytest.approx(fd, rel=GRAD_REL, abs=GRAD_ABS)
    for i in np.argsort(-np.abs(ref["dcost"]))[:3]:
        e = np.zeros_like(cost)
        e[i] = h
        fd = (val(c=cost + e) - val(c=cost - e)) / (2 * h)
        assert dc[i] == pytest.approx(fd, rel=GRAD_REL, abs=1e-8)


def test_autograd_gradients_of_b0_and_accuracy(api):
    """QVRootValue with b0 as an input and a belief that straddles label
    regions: every gradient torch returns against the oracle's reverse mode."""
    from paper_1810_00204_gb300.autograd import root_value
    w = _spread(_with_cost(WL.tiny(8), 8))
    S = 50
    slip = torch.tensor(float(w.slip), dtype=torch.float32, requires_grad=True)
    acc = torch.tensor(float(w.accuracy), dtype=torch.float32, requires_grad=True)
    cost = torch.from_numpy(w.cost.copy()).requires_grad_(True)
    b0 = torch.from_numpy(w.b0.copy()).requires_grad_(True)
    # the oracle's own draws, replayed into the GPU plan
    p = _prob(w)
    rep = O.tree_plan(p, O.value_iteration(p, truncated=S)["Q"], depth=2, K=6, seed=w.seed,
                      episode=w.episode)["samples_flat"]
    v = root_value(w, slip, acc, cost, b0, depth=2, K=6, seed=w.seed, episode=w.episode, sweeps=S, every=7,
                   replay=torch.from_numpy(rep.copy()).cuda())
    gs, ga, gc, gb = torch.autograd.grad(v, (slip, acc, cost, b0))
    assert gs.dtype == torch.float32 and gc.shape == cost.shape and gb.device == b0.device
    ref = O.root_value_grad(p, S, depth=2, K=6, replay=rep)
    assert float(gs) == pytest.approx(ref["dslip"], rel=GRAD_REL)
    assert float(ga) == pytest.approx(ref["dacc"], rel=GRAD_REL, abs=GRAD_ABS)
    assert abs(ref["dacc"]) > 1e3 * GRAD_ABS
    _close(gc.numpy().ravel(), ref["dcost"], GRAD_REL, what="dcost")
    _close(gb.numpy().ravel(), ref["db0"], GRAD_REL, what="db0")
