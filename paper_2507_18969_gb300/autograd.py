"""torch.autograd.Function around the library's hand-written adjoint.

The online update of Algorithm 1 (loss.backward() on the cross-entropy of
Eq. 2, then an optimizer step) runs inside the library. This wrapper exposes
that same forward and adjoint to autograd, so a caller can check the
gradient with torch tools (for example against finite differences) or drive
the model from PyTorch. The forward and backward here only marshal tensors:
the forward pass, the softmax and the adjoint are the library's kernels
(edpc_model_forward and edpc_model_backward).
"""
from __future__ import annotations

import numpy as np
import torch

from . import Model


class EDPCStepLoss(torch.autograd.Function):
    """Mean cross-entropy over the active streams at a given state.

    Inputs: ``shared`` (param_count FP32, canonical order) and ``fdm``
    (streams x F' x F' FP32), both CPU tensors; a ``Model`` handle; and the
    step's ``ctx`` (streams x K uint8), ``targets`` (streams) and ``active``
    (streams, 0/1). Returns a 0-d FP32 tensor. Gradients flow to ``shared``
    and ``fdm``.
    """

    @staticmethod
    def forward(ctx, shared, fdm, model: Model, contexts, targets, active):
        model.set_state(P=shared.detach().cpu().numpy(), U=fdm.detach().cpu().numpy())
        c = np.ascontiguousarray(contexts, dtype=np.uint8)
        tg = np.ascontiguousarray(targets, dtype=np.uint8)
        ac = np.ascontiguousarray(active, dtype=np.uint8)
        _, p = model.forward(c)
        rows = np.nonzero(ac)[0]
        loss = float(-np.log(p[rows, tg[rows]].astype(np.float64)).mean()) if rows.size else 0.0
        ctx.model, ctx.c, ctx.tg, ctx.ac = model, c, tg, ac
        return torch.tensor(loss, dtype=torch.float32)

    @staticmethod
    def backward(ctx, gout):
        g, gu = ctx.model.backward(ctx.c, ctx.tg, ctx.ac)
        gs = torch.from_numpy(g) * gout
        gf = torch.from_numpy(gu) * gout
        return gs, gf, None, None, None, None


def step_loss(shared, fdm, model: Model, contexts, targets, active):
    return EDPCStepLoss.apply(shared, fdm, model, contexts, targets, active)
