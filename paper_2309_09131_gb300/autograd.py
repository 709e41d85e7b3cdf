"""``torch.autograd.Function`` wrappers over the C ABI.

* ``SpMTTKRP``: M = spMTTKRP_mode(X, factors); its backward is the adjoint
  kernel path (``flycoo_mttkrp_adjoint``): dY_w = spMTTKRP_w with the output
  mode's factor replaced by the upstream gradient, one fused pass per mode
  in that mode's own FLYCOO layout.
* ``CPOPTLoss``: weighted CP on the observed entries,
  L = 1/2 sum_x (x - m_x)^2 with m_x the CPD model value (Eq. 1); the forward
  runs ``flycoo_cpopt_grad`` (loss and all factor gradients in one sweep) and
  the backward scales the stored gradients.

The tensor's nonzero values are data, not parameters: neither function
returns a gradient for them.  Factors must be FP32 CUDA tensors.
"""
from __future__ import annotations

from typing import Sequence

import torch

from . import _native as nat


class SpMTTKRP(torch.autograd.Function):
    @staticmethod
    def forward(ctx, T, mode: int, *factors):
        if T.layout_mode != mode:
            nat.flycoo_remap(T.h, mode)
        R = next(f.shape[1] for w, f in enumerate(factors) if w != mode)
        out = torch.empty((T.dims[mode], R), dtype=torch.float32, device=factors[0].device)
        nat.flycoo_spmttkrp(T.h, mode, factors, out, (mode + 1) % T.N)
        ctx.T = T
        ctx.mode = mode
        ctx.save_for_backward(*factors)
        return out

    @staticmethod
    def backward(ctx, G):
        factors = ctx.saved_tensors
        mode = ctx.mode
        grads = [None] * len(factors)
        want = [w != mode and ctx.needs_input_grad[2 + w] for w in range(len(factors))]
        if any(want):
            grads = [torch.empty_like(f) if want[w] else None for w, f in enumerate(factors)]
            nat.flycoo_mttkrp_adjoint(ctx.T.h, mode, factors, G.contiguous().float(), grads)
        return (None, None, *grads)


def spmttkrp(T, mode: int, factors: Sequence[torch.Tensor]) -> torch.Tensor:
    """Differentiable spMTTKRP of ``mode``."""
    return SpMTTKRP.apply(T, mode, *factors)


class CPOPTLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, T, *factors):
        grads = [torch.empty_like(f) for f in factors]
        loss = nat.flycoo_cpopt_grad(T.h, factors, grads)
        ctx.save_for_backward(*grads)
        return torch.tensor(loss, dtype=torch.float64, device=factors[0].device)

    @staticmethod
    def backward(ctx, gL):
        grads = ctx.saved_tensors
        return (None, *[g * gL.to(g.dtype) for g in grads])


def cpopt_loss(T, factors: Sequence[torch.Tensor]) -> torch.Tensor:
    """Differentiable CP-OPT loss 1/2 sum over the nonzeros of (x - m_x)^2."""
    return CPOPTLoss.apply(T, *factors)
