"""``torch.autograd.Function`` over the library's forward (itc_run with no iterations: fields,
S_XX and D_cs of Eq. (1)) and its hand-written adjoint (itc_backward).  Glue only: both passes
run in libitc.so's kernels."""
from __future__ import annotations

import torch

from . import itc


class ITCDivergence(torch.autograd.Function):
    """D_cs per image for a batch of 2-D weight images h_b (float32 [H_b, W_b], CUDA) and codebooks
    W_b (float32 [M_b, 2]).  Call as ``ITCDivergence.apply(sigma, trunc, *hs, *Ws)``; returns a
    float32 tensor [B].  Gradients flow to every h_b and W_b (weighted ITC, Sec. 5)."""

    @staticmethod
    def forward(ctx, sigma, trunc, *tensors):
        B = len(tensors) // 2
        hs, Ws = tensors[:B], tensors[B:]
        dev = hs[0].device
        plan = itc.Plan([h.detach() for h in hs], [int(w.shape[0]) for w in Ws], itc.make_params(sigma, trunc, 0))
        W = torch.cat([w.detach().reshape(-1).float() for w in Ws]).contiguous()
        st = itc.new_stats(B, dev)
        itc.run(plan, W, st)
        ctx.plan, ctx.W = plan, W
        ctx.shapes = [tuple(w.shape) for w in Ws]
        return st.view(torch.float64).view(B, 7)[:, 0].float()

    @staticmethod
    def backward(ctx, grad):
        plan, W = ctx.plan, ctx.W
        gW = torch.empty_like(W)
        gh = torch.empty(plan.pixels, dtype=torch.float32, device=W.device)
        itc.backward(plan, W, grad_dcs=grad.float().contiguous(), grad_W=gW, grad_h=gh)
        ghs = [gh[plan.gh_offsets[b]:plan.gh_offsets[b + 1]].view(plan.shapes[b]) for b in range(plan.B)]
        gWs = [gW[plan.w_offsets[b]:plan.w_offsets[b + 1]].view(ctx.shapes[b]) for b in range(plan.B)]
        return (None, None, *ghs, *gWs)
