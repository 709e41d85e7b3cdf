"""``torch.autograd.Function`` wrappers over the C ABI.

* ``SpMTTKRP``: M = spMTTKRP_mode(X, factors); its backward is the adjoint
  kernel path (``flycoo_mttkrp_adjoint``): dY_w = spMTTKRP_w with the output
  mode's factor replaced by the upstream gradient, one fused pass per mode
  in that mode's own FLYCOO layout, and, when the values are passed in and
  require a gradient, d val(x) = the CP model value at x with the output
  mode's factor replaced by the upstream gradient.
* ``CPOPTLoss``: weighted CP on the observed entries,
  L = 1/2 sum_x (x - m_x)^2 with m_x the CPD model value (Eq. 1); the forward
  runs ``flycoo_cpopt_grad`` (loss and all factor gradients in one sweep) and
  the backward scales the stored gradients.

``SpMTTKRP`` takes FP32 or BF16 factors (BF16 factors get BF16 upstream
gradients in the backward, FP32 accumulation); ``CPOPTLoss`` takes FP32.
"""
from __future__ import annotations

from typing import Sequence

import torch

from . import _native as nat


class SpMTTKRP(torch.autograd.Function):
    @staticmethod
    def forward(ctx, T, mode: int, vals, *factors):
        if T.layout_mode != mode:
            nat.flycoo_remap(T.h, mode)
        R = next(f.shape[1] for w, f in enumerate(factors) if w != mode)
        out = torch.empty((T.dims[mode], R), dtype=torch.float32, device=factors[0].device)
        nat.flycoo_spmttkrp(T.h, mode, factors, out, (mode + 1) % T.N)
        ctx.T = T
        ctx.mode = mode
        ctx.has_vals = vals is not None
        ctx.save_for_backward(*factors)
        return out

    @staticmethod
    def backward(ctx, G):
        factors = ctx.saved_tensors
        mode = ctx.mode
        dt = next(f.dtype for w, f in enumerate(factors) if w != mode)
        grads = [None] * len(factors)
        want = [w != mode and ctx.needs_input_grad[3 + w] for w in range(len(factors))]
        want_vals = ctx.has_vals and ctx.needs_input_grad[2]
        gvals = None
        if any(want) or want_vals:
            out = [torch.empty(f.shape, dtype=torch.float32, device=f.device) if want[w] else None
                   for w, f in enumerate(factors)]
            if want_vals:
                gvals = torch.empty(ctx.T.nnz, dtype=torch.float32, device=G.device)
            nat.flycoo_mttkrp_adjoint(ctx.T.h, mode, factors, G.contiguous().to(dt), out, gvals)
            grads = [o.to(f.dtype) if o is not None else None for o, f in zip(out, factors)]
        return (None, None, gvals, *grads)


def spmttkrp(T, mode: int, factors: Sequence[torch.Tensor], vals=None) -> torch.Tensor:
    """Differentiable spMTTKRP of ``mode``.  ``vals``, when given, stands for
    the tensor's nonzero values in the COO order ``T`` was created from (it
    must hold those values); a gradient for it is then returned by the
    backward pass."""
    return SpMTTKRP.apply(T, mode, vals, *factors)


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
