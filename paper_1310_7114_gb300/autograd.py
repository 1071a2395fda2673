"""``torch.autograd.Function`` over the library's forward (itc_run with no iterations: fields,
S_XX and D_cs of Eq. (1)) and its hand-written adjoint (itc_backward).  Glue only: both passes
run in libitc.so's kernels.

The fields of a batch take 12 bytes per pixel.  When they fit in device memory the forward keeps
them (the plan's workspace) for the backward.  When they do not, or when the caller sets a fields
budget, neither pass keeps them: the forward and the backward each recompute them image range by
image range inside a window of the budget's size (itc_run_budget, itc_backward_budget), with the
same results bit for bit."""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import itc

# share of the free device memory the stored fields may take before the recomputing path is used
_STORE_FRACTION = 0.5


def _forward(ctx, sigma, trunc, budget: Optional[int], tensors):
    B = len(tensors) // 2
    hs, Ws = tensors[:B], tensors[B:]
    dev = hs[0].device
    plan = itc.Plan([h.detach() for h in hs], [int(w.shape[0]) for w in Ws], itc.make_params(sigma, trunc, 0),
                    allocate_ws=False)
    if budget is None:
        # whole-batch fields only if they fit comfortably in what the device has free
        free, _ = torch.cuda.mem_get_info(dev)
        if plan.ws_bytes > _STORE_FRACTION * free:
            budget = int(_STORE_FRACTION * free)
        else:
            plan.ws = torch.empty(max(plan.ws_bytes, 256), dtype=torch.uint8, device=dev)
    W = torch.cat([w.detach().reshape(-1).float() for w in Ws]).contiguous()
    st = itc.new_stats(B, dev)
    if budget is None:
        itc.run(plan, W, st)
        ctx.ws = None
    else:
        ctx.ws = itc.budget_workspace(plan, int(budget))
        itc.run_budget(plan, W, ctx.ws, st)
    ctx.plan, ctx.W = plan, W
    ctx.shapes = [tuple(w.shape) for w in Ws]
    return st.view(torch.float64).view(B, 7)[:, 0].float()


def _backward(ctx, grad):
    plan, W = ctx.plan, ctx.W
    gW = torch.empty_like(W)
    gh = torch.empty(plan.pixels, dtype=torch.float32, device=W.device)
    if ctx.ws is None:
        itc.backward(plan, W, grad_dcs=grad.float().contiguous(), grad_W=gW, grad_h=gh)
    else:
        itc.backward_budget(plan, W, ctx.ws, grad_dcs=grad.float().contiguous(), grad_W=gW, grad_h=gh)
    ghs = [gh[plan.gh_offsets[b]:plan.gh_offsets[b + 1]].view(plan.shapes[b]) for b in range(plan.B)]
    gWs = [gW[plan.w_offsets[b]:plan.w_offsets[b + 1]].view(ctx.shapes[b]) for b in range(plan.B)]
    return ghs, gWs


class ITCDivergence(torch.autograd.Function):
    """D_cs per image for a batch of 2-D weight images h_b (float32 [H_b, W_b], CUDA) and codebooks
    W_b (float32 [M_b, 2]).  Call as ``ITCDivergence.apply(sigma, trunc, *hs, *Ws)``; returns a
    float32 tensor [B].  Gradients flow to every h_b and W_b (weighted ITC, Sec. 5).  The fields
    are kept between the passes when they fit in half the free device memory, else recomputed."""

    @staticmethod
    def forward(ctx, sigma, trunc, *tensors):
        return _forward(ctx, sigma, trunc, None, tensors)

    @staticmethod
    def backward(ctx, grad):
        ghs, gWs = _backward(ctx, grad)
        return (None, None, *ghs, *gWs)


class ITCDivergenceBudget(torch.autograd.Function):
    """ITCDivergence with a fields budget in bytes: ``ITCDivergenceBudget.apply(sigma, trunc,
    budget_bytes, *hs, *Ws)``.  The workspace the two passes share is about budget_bytes (at
    least the fields of the largest image plus a few bytes per image and tile); the fields are
    recomputed range by range in both passes."""

    @staticmethod
    def forward(ctx, sigma, trunc, budget_bytes, *tensors):
        return _forward(ctx, sigma, trunc, int(budget_bytes), tensors)

    @staticmethod
    def backward(ctx, grad):
        ghs, gWs = _backward(ctx, grad)
        return (None, None, None, *ghs, *gWs)


def itc_divergence(hs: Sequence[torch.Tensor], Ws: Sequence[torch.Tensor], sigma, trunc: float = 3.0,
                   fields_budget_bytes: Optional[int] = None) -> torch.Tensor:
    """D_cs per image with autograd; ``fields_budget_bytes`` forces the recomputing path."""
    if fields_budget_bytes is None:
        return ITCDivergence.apply(sigma, trunc, *hs, *Ws)
    return ITCDivergenceBudget.apply(sigma, trunc, int(fields_budget_bytes), *hs, *Ws)
