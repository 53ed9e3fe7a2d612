"""torch.autograd wrapper of the forward map and its hand-written adjoint.

UltimaRatioIQ.apply(cell, weights, plan, shape, origin) -> mean I per Q bin
(float64 [B], NaN for empty bins), computed by ur_fft_intensity_tiled; the
backward pass is ur_backward, which recomputes the spectrum column by column
from the forward intermediate kept in the workspace, scales it by
2 dL/dmean_j / n_j, inverts the transform and reduces over the tiling into
dL/d cell and (when `weights` is a tensor) dL/d weights.  Both passes run in
libur's kernels.

The workspace is the plan's own (Plan.claim_workspace), allocated once and
reused by every call.  When another forward has claimed it between a forward
and its backward, the backward first re-runs that forward's plane pass into
it (the intermediate is a deterministic function of the inputs).
"""
from __future__ import annotations

import torch

from . import api


class UltimaRatioIQ(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cell: torch.Tensor, weights, plan: api.Plan, shape, origin=(0, 0, 0)):
        cell = cell.contiguous()
        if weights is not None:
            weights = weights.contiguous()
            from .inputs import SHAPE_WEIGHTS, Shape
            shape = Shape(SHAPE_WEIGHTS)
        ws, gen = plan.claim_workspace(api.UR_WS_FORWARD | api.UR_WS_BACKWARD, device=cell.device)
        bins = api.fft_intensity_tiled(plan, cell, shape, origin=origin, weights=weights, ws=ws)
        ctx.plan, ctx.shape, ctx.origin, ctx.gen = plan, shape, origin, gen
        ctx.has_weights = weights is not None
        ctx.save_for_backward(cell, weights if weights is not None else torch.empty(0, device=cell.device), bins)
        return bins[api.BIN_MEAN].clone()

    @staticmethod
    def backward(ctx, g_mean):
        cell, weights, bins = ctx.saved_tensors
        weights = weights if ctx.has_weights else None
        g = torch.where(bins[api.BIN_COUNT] > 0, torch.nan_to_num(g_mean.to(torch.float64)), 0.0).contiguous()
        want_mask = ctx.has_weights and ctx.needs_input_grad[1]
        plan = ctx.plan
        if plan.workspace_generation() != ctx.gen:
            # another forward wrote the shared workspace since: restore this one's intermediate
            ws, ctx.gen = plan.claim_workspace(api.UR_WS_FORWARD | api.UR_WS_BACKWARD, device=cell.device)
            api.fft_intensity_tiled(plan, cell, ctx.shape, origin=ctx.origin, weights=weights, ws=ws,
                                    want_bins=False)
        ws = plan._ws
        dcell, dmask = api.backward(plan, g, bins, cell, ctx.shape, ws, origin=ctx.origin, weights=weights,
                                    want_mask=want_mask)
        return dcell, (dmask if want_mask else None), None, None, None


def binned_intensity(cell: torch.Tensor, plan: api.Plan, shape, weights: torch.Tensor | None = None,
                     origin=(0, 0, 0)) -> torch.Tensor:
    """Differentiable Sec. 2.3-2.5 forward: mean I(Q) per bin (float64, Eq. 1 normalisation)."""
    return UltimaRatioIQ.apply(cell, weights, plan, shape, origin)
