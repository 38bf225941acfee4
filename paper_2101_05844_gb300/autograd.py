"""torch.autograd.Function over the Active Set bound and its envelope gradient.

`ActiveSetBound.apply(context, lo, hi, W_1, b_1, ..., W_n, b_n)` returns the bound of every
subproblem (float64, on lo's device) at the context's current duals; its backward calls
`as_bound_backward`, the gradient at fixed duals, masks, intermediate bounds and signs of W
(Danskin), with respect to the weights, biases (of the last layer through the property rows) and
the input box. The context holds its own copies of the weights (made by `as_init`) and of the box
(`as_init`, `as_reset`); the tensors passed here must hold the same values and serve as the leaves
the gradient is attached to. Tensors holding other values (a training loop that updated the
weights, a new box) are refused with an error rather than given the gradient of the context's
stale copies: build a new context (weights) or reset it and iterate (box) first.
"""
from __future__ import annotations

import numpy as np
import torch


class ActiveSetBound(torch.autograd.Function):
    @staticmethod
    def forward(ctx, context, lo, hi, *params):
        why = context.holds(lo, hi, params)
        if why is not None:
            raise ValueError(f"ActiveSetBound: {why}; the bound and its gradient would belong to other values")
        ctx.context = context
        ctx.save_for_backward(lo, hi, *params)
        out = torch.zeros(context.S, dtype=torch.float64, device=lo.device)
        context.bound_into(64, out)
        return out

    @staticmethod
    def backward(ctx, grad):
        lo, hi, *params = ctx.saved_tensors
        dev = lo.device
        g = grad.detach().to(torch.float64).contiguous()
        if g.device.type != "cuda":
            g = g.to(dev)
        dW = [torch.zeros_like(p, dtype=torch.float32, device=dev) for p in params[0::2]]
        db = [torch.zeros_like(p, dtype=torch.float32, device=dev) for p in params[1::2]]
        dlo = torch.zeros_like(lo, dtype=torch.float32, device=dev)
        dhi = torch.zeros_like(hi, dtype=torch.float32, device=dev)
        ctx.context.backward(g, dW, db, dlo, dhi)
        grads = []
        for w, b in zip(dW, db):
            grads += [w, b]
        return (None, dlo.to(lo.dtype), dhi.to(hi.dtype), *[q.to(p.dtype) for q, p in zip(grads, params)])


def bound(context, lo, hi, params):
    """Differentiable bounds [S]; params = [W_1, b_1, ..., W_n, b_n] (CUDA tensors)."""
    return ActiveSetBound.apply(context, lo, hi, *params)
