"""torch.autograd.Function around the library's decoder training pass.

``decoder_uJ(trainer, q, params)`` returns u = D(q) (B, N) and J = dD/dq (B, N, r)
for a batch of latents, with the backward (w.r.t. q and every weight and bias)
computed by the library's hand-written reverse sweep (``dae_train_backward``):
split-BF16x3 tensor-core GEMMs, activations checkpointed every second layer.
PyTorch only holds the tensors; every step of the pass runs in the library.
"""
from __future__ import annotations

import torch

from . import dae


class _DecoderUJ(torch.autograd.Function):
    @staticmethod
    def forward(ctx, trainer, q, *params):
        W, b = list(params[0::2]), list(params[1::2])
        B, r = q.shape
        N = W[-1].shape[0]
        qd = q.detach().to(torch.float64).contiguous()
        uJ = torch.empty((1 + r, B, N), device=q.device, dtype=torch.float32)
        dae.dae_train_forward(trainer, [w.detach().contiguous() for w in W],
                              [x.detach().contiguous() for x in b], qd, uJ)
        ctx.trainer = trainer
        ctx.save_for_backward(qd, *params)
        ctx.q_dtype = q.dtype
        return uJ[0].clone(), uJ[1:].permute(1, 2, 0).contiguous()

    @staticmethod
    def backward(ctx, gu, gJ):
        qd, *params = ctx.saved_tensors
        W, b = list(params[0::2]), list(params[1::2])
        B, r = qd.shape
        N = W[-1].shape[0]
        g_uJ = torch.zeros((1 + r, B, N), device=qd.device, dtype=torch.float32)
        if gu is not None:
            g_uJ[0] = gu
        if gJ is not None:
            g_uJ[1:] = gJ.permute(2, 0, 1)
        gW = [torch.empty_like(w) for w in W]
        gb = [torch.empty_like(x) for x in b]
        gq = torch.empty_like(qd)
        dae.dae_train_backward(ctx.trainer, [w.detach().contiguous() for w in W],
                               [x.detach().contiguous() for x in b], qd, g_uJ, gq, gW, gb)
        grads = []
        for a, c in zip(gW, gb):
            grads += [a, c]
        return (None, gq.to(ctx.q_dtype), *grads)


def decoder_uJ(trainer, q, params):
    """u (B, N) and J (B, N, r) of the decoder with parameters [W0, b0, W1, b1, ...]."""
    return _DecoderUJ.apply(trainer, q, *params)
