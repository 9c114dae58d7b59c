"""The plan's root value as a differentiable PyTorch function.

`QVRootValue` wraps the C ABI: its forward runs the checkpointed FP64 value
iteration (mdp_value_iterate_checkpointed) and one plan (qv_plan_run); its
backward runs qv_tree_backward and mdp_value_backward, which return the
derivatives of the root value U_V(b0) with respect to the slip, the sensor
accuracy, the per-cell cost map and b0.  The sampled measurements, the FREQ
weights and every max are those of the forward pass (held fixed), as for any
piecewise-smooth function.  Argument marshalling only: every step runs in the
CUDA library.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import _native as N
from . import api


class QVRootValue(torch.autograd.Function):
    """root = QVRootValue.apply(slip, accuracy, cost, b0, workload, depth, K,
    seed, episode, sweeps, every, leaf_mode, replay)

    slip, accuracy: 0-dim tensors; cost: [H, W] tensor or None (no cost map);
    b0: [H, W] tensor or None (the workload's b0); replay: None, or int32
    observation samples on the device to use instead of the Philox draws
    (laid out as qv_plan_params_t.d_replay).  Returns a 0-dim FP64 tensor on
    the CUDA device.  Gradients come back in the inputs' dtypes."""

    @staticmethod
    def forward(ctx, slip, accuracy, cost, b0, w, depth, K, seed, episode, sweeps, every, leaf_mode, replay=None):
        dev = torch.device("cuda")
        c = None if cost is None else cost.detach().to(dev, torch.float32)
        model = api.Model(w, device=dev, slip=float(slip), accuracy=float(accuracy), cost=c)
        vi = api.mdp_value_iterate_checkpointed(model, sweeps, every)
        b0g = model.b0() if b0 is None else model.to_grid(b0.detach().to(dev, torch.float32))
        lm = N.QV_LEAF_MATERIALISE if leaf_mode == "materialise" else N.QV_LEAF_FUSED
        plan = api.Plan([model], [vi["Q"]], [b0g], depth, K, seed, episode, N.QV_WEIGHT_FREQ, lm, replay)
        plan.run()
        r = plan.read()[0]
        ctx.state = (model, vi, plan, b0g)
        ctx.meta = (slip, accuracy, cost, b0)
        ctx.result = r
        return torch.tensor(r["value"], dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, g):
        model, vi, plan, _ = ctx.state
        slip, accuracy, cost, b0 = ctx.meta
        tb = api.qv_tree_backward(plan, 0, dL=float(g), want_db0=b0 is not None and ctx.needs_input_grad[3])
        api.mdp_value_backward(model, vi, tb["Qbar"], tb["dslip"], tb["dcost"])
        W = model.W
        d_slip = tb["dslip"][0].to(slip.dtype).to(slip.device) if ctx.needs_input_grad[0] else None
        d_acc = tb["dacc"][0].to(accuracy.dtype).to(accuracy.device) if ctx.needs_input_grad[1] else None
        d_cost = None
        if cost is not None and ctx.needs_input_grad[2]:
            d_cost = tb["dcost"][:, :W].reshape(cost.shape).to(cost.dtype).to(cost.device)
        d_b0 = None
        if b0 is not None and ctx.needs_input_grad[3]:
            d_b0 = tb["db0"][:, :W].reshape(b0.shape).to(b0.dtype).to(b0.device)
        return (d_slip, d_acc, d_cost, d_b0) + (None,) * 9


def root_value(w, slip: torch.Tensor, accuracy: torch.Tensor, cost: Optional[torch.Tensor] = None,
               b0: Optional[torch.Tensor] = None, depth: int = 3, K: int = 8, seed: int = 0, episode: int = 0,
               sweeps: int = 200, every: int = 16, leaf_mode: str = "fused",
               replay: Optional[torch.Tensor] = None) -> torch.Tensor:
    """U_V(b0) of one plan on the map of workload `w`, differentiable in
    slip, accuracy, cost and b0 (replay: fixed observation samples)."""
    return QVRootValue.apply(slip, accuracy, cost, b0, w, depth, K, seed, episode, sweeps, every, leaf_mode, replay)
