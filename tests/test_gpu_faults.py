"""Failure detection without a GPU fault: with QVTS_FAULT=timeout the host
passes a poll limit of 0 to every wait on other CTAs (grid barrier, progress
flags), so the first wait that is not already satisfied gives up, sets the
status word and every CTA leaves.  The call must report QV_ERR_TIMEOUT, the
context must stay usable, and the next call without the fault must give the
normal result."""
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


def test_plan_timeout_is_reported_and_the_plan_recovers(api, monkeypatch):
    from paper_1810_00204_gb300 import _native as N
    w = WL.tiny(0)
    m = api.Model(w)
    Qo = O.value_iteration(w)["Q"].astype(np.float32)  # the oracle's Q feeds both sides
    Q = m.to_grid(Qo.reshape(5, w.H, w.W))
    p = api.Plan([m], [Q], [m.b0()], depth=w.depth, K=w.K, seed=w.seed)
    p.run()
    ref = p.read()[0]
    monkeypatch.setenv("QVTS_FAULT", "timeout")
    p.run()
    with pytest.raises(N.QVError) as ei:
        p.read()
    assert ei.value.status == N.QV_ERR_TIMEOUT
    monkeypatch.delenv("QVTS_FAULT")
    assert torch.ones(4, device="cuda").sum().item() == 4.0  # the context is usable
    p.run()
    got = p.read()[0]
    assert got["nodes_per_level"] == ref["nodes_per_level"]
    assert got["value"] == ref["value"] and got["action"] == ref["action"]
    o = O.tree_plan(w, Qo.astype(np.float64))
    assert abs(got["value"] - o["root_value"]) <= 1e-5 * max(1.0, abs(o["root_value"]))


@pytest.mark.parametrize("truncated", [0, 50])
def test_value_iteration_timeout_is_reported(api, monkeypatch, truncated):
    from paper_1810_00204_gb300 import _native as N
    w = WL.mid(0)
    m = api.Model(w)
    monkeypatch.setenv("QVTS_FAULT", "timeout")
    with pytest.raises(N.QVError) as ei:
        api.mdp_value_iterate(m, dtype="f32", truncated=truncated)
    assert ei.value.status == N.QV_ERR_TIMEOUT
    monkeypatch.delenv("QVTS_FAULT")
    vi = api.mdp_value_iterate(m, dtype="f32", truncated=truncated)
    assert vi["status"] == N.QV_OK
    assert vi["sweeps"] == (truncated if truncated else vi["sweeps"]) and vi["sweeps"] > 0


def test_value_iteration_adjoint_timeout_is_reported(api, monkeypatch):
    from paper_1810_00204_gb300 import _native as N
    w = WL.diff(0)
    m = api.Model(w)
    vi = api.mdp_value_iterate_checkpointed(m, 40, 16)
    Qbar = torch.ones((5, m.H, m.P), dtype=torch.float64, device="cuda")
    dslip = torch.zeros(1, dtype=torch.float64, device="cuda")
    dcost = torch.zeros((m.H, m.P), dtype=torch.float64, device="cuda")
    monkeypatch.setenv("QVTS_FAULT", "timeout")
    with pytest.raises(N.QVError) as ei:
        api.mdp_value_backward(m, vi, Qbar, dslip, dcost)
    assert ei.value.status == N.QV_ERR_TIMEOUT
    monkeypatch.delenv("QVTS_FAULT")
    dslip.zero_()
    dcost.zero_()
    api.mdp_value_backward(m, vi, Qbar, dslip, dcost)
    ref = O.vi_backward(O.Problem(w, slip=float(w.slip), accuracy=float(w.accuracy), discount=float(w.discount),
                                  cost=w.cost.astype(np.float64).ravel()), 40,
                        m.from_grid(Qbar).reshape(5, -1))
    assert float(dslip[0]) == pytest.approx(ref["dslip"], rel=1e-9)


@pytest.mark.parametrize("mode,status", [("oom", "QV_ERR_WORKSPACE"), ("invalid", "QV_ERR_INVALID")])
def test_injected_host_faults_and_recovery(api, monkeypatch, mode, status):
    """QVTS_FAULT=oom|invalid: the value iteration, the plan's creation and
    the Bayes correction report the injected status with a message naming
    it, and the same calls succeed once the variable is unset."""
    from paper_1810_00204_gb300 import _native as N
    code = getattr(N, status)
    w = WL.tiny(2)
    m = api.Model(w)
    Qo = O.value_iteration(w)["Q"].astype(np.float32)  # the oracle's Q feeds both sides
    Q = m.to_grid(Qo.reshape(5, w.H, w.W))
    b = m.b0()
    monkeypatch.setenv("QVTS_FAULT", mode)
    for call in (lambda: api.mdp_value_iterate(m, dtype="f32"),
                 lambda: api.Plan([m], [Q], [b], depth=w.depth, K=w.K, seed=w.seed),
                 lambda: api.belief_correct(m, b, 0)):
        with pytest.raises(N.QVError) as ei:
            call()
        assert ei.value.status == code
        assert f"QVTS_FAULT={mode}".encode() in N.lib().qv_last_error()
    monkeypatch.delenv("QVTS_FAULT")
    assert api.mdp_value_iterate(m, dtype="f32")["status"] == N.QV_OK
    p = api.Plan([m], [Q], [b], depth=w.depth, K=w.K, seed=w.seed)
    p.run()
    r = p.read()[0]
    o = O.tree_plan(w, Qo.astype(np.float64))
    assert abs(r["value"] - o["root_value"]) <= 1e-5 * max(1.0, abs(o["root_value"]))
    out, pz = api.belief_correct(m, b, 0)
    assert torch.isfinite(out).all()
