"""torch.autograd.Function over the PWF forward model (Eq. (1)).

forward:  f = f(psi, t) of Eq. (1)                      -> pwf_forward
backward: (dL/dpsi, dL/dt) for a real cotangent dL/df    -> pwf_forward_vjp

Only psi and t are saved for the backward pass; the propagated fields (P1{x},
the detector field v) are recomputed inside pwf_forward_vjp rather than
stored, which keeps the memory of a batch at a few fields per projection.
Gradients follow PyTorch's convention for complex inputs of a real loss:
dL/dRe + i dL/dIm.
"""
from __future__ import annotations

import torch

from . import pwf as _pwf


def _aligned(x: torch.Tensor) -> torch.Tensor:
    """x as a contiguous tensor whose data starts on a 16-byte boundary (the
    library's rule for device arrays): a fresh copy when a view starts in
    between. Inputs only: the copy is never written back."""
    x = x.contiguous()
    return x if x.data_ptr() % 16 == 0 else x.clone()


class PWFForward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi: torch.Tensor, t: torch.Tensor, plan: "_pwf.Plan"):
        if psi.dtype != torch.complex64 or t.dtype != torch.complex64:
            raise TypeError("psi and t must be complex64")
        psi = _aligned(psi)
        t = _aligned(t)
        f = plan.forward(psi, t)
        ctx.save_for_backward(psi, t)
        ctx.plan = plan
        return f

    @staticmethod
    def backward(ctx, grad_f: torch.Tensor):
        psi, t = ctx.saved_tensors
        want_psi, want_t = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        gp, gt = ctx.plan.vjp(psi, t, _aligned(grad_f.to(torch.float32)), want_psi=want_psi, want_t=want_t)
        return gp, gt, None


def physical_model(psi: torch.Tensor, t: torch.Tensor, plan: "_pwf.Plan") -> torch.Tensor:
    """Differentiable forward model f(psi, t) of Eq. (1) on the CUDA path."""
    return PWFForward.apply(psi, t, plan)
