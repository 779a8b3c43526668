"""torch.autograd.Functions over the library's field and energy kernels.

* ``DemagField.apply(M, plan)``: H = -N * M; the backward pass applies the
  adjoint kernel path (``demag_field_adjoint``) to the incoming gradient. The
  tensor is symmetric and even, so the adjoint is another field evaluation.
* ``DemagEnergy.apply(m, Ms, w, plan)``: E = -(mu0/2) V sum M.H for
  M = Ms * w * m (paper Sec. 2). Nothing is saved between forward and
  backward beyond the inputs: the backward pass re-runs the pipeline
  (checkpointing of the padded spectra) with the gradient epilogue,
  dE/dm = -mu0 V Ms w H, scaled on the device by the upstream gradient.
"""
from __future__ import annotations

import torch


class DemagField(torch.autograd.Function):
    @staticmethod
    def forward(ctx, M, plan):
        ctx.plan = plan
        return plan.field(M)

    @staticmethod
    def backward(ctx, gH):
        return ctx.plan.field_adjoint(gH.contiguous()), None


class DemagEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, Ms, w, plan):
        ctx.plan = plan
        ctx.Ms = float(Ms)
        ctx.has_w = w is not None
        ctx.save_for_backward(m, w) if w is not None else ctx.save_for_backward(m)
        E, _ = plan.energy_grad(m, Ms, w, want_energy=True, want_grad=False)
        return E

    @staticmethod
    def backward(ctx, gE):
        saved = ctx.saved_tensors
        m = saved[0]
        w = saved[1] if ctx.has_w else None
        g = gE.detach().to(dtype=torch.float64).reshape(()).contiguous()
        _, grad = ctx.plan.energy_grad(m, ctx.Ms, w, want_energy=False, want_grad=True, gscale=g)
        return grad, None, None, None


def demag_field(M, plan):
    return DemagField.apply(M, plan)


def demag_energy(m, Ms, plan, w=None):
    return DemagEnergy.apply(m, Ms, w, plan)
