"""torch.autograd.Function around the library's E-step means and their adjoint.

forward(Phi, y, alpha) runs one E-step on the GPU (cmcs_set_data, cmcs_set_alpha,
cmcs_estep) and returns the posterior means mu [T][C][D]; backward(dL/dmu) calls
cmcs_adjoint, one extra batched solve with the same symmetric operator, and returns dL/dPhi,
dL/dy and dL/dalpha.  Responsibilities, s and the log-det estimate are constants for the
derivative.  Between forward and backward the context must not run another E-step."""
from __future__ import annotations

import torch

from . import cmcs


class PosteriorMeans(torch.autograd.Function):
    @staticmethod
    def forward(ctx, context: "cmcs.Context", Phi, y, alpha, em_iter: int = 0):
        context.set_data(Phi.detach().contiguous(), y.detach().contiguous())
        context.set_alpha(alpha.detach().contiguous(), int(em_iter))
        context.estep()
        ctx.context = context
        return context.read(cmcs.OUT_MU, device=True)

    @staticmethod
    def backward(ctx, g):
        dy, dalpha, dPhi = ctx.context.adjoint(g.contiguous().float())
        return None, dPhi, dy, dalpha, None


def posterior_means(context, Phi, y, alpha, em_iter: int = 0):
    """mu = PosteriorMeans.apply(...), differentiable with respect to Phi, y and alpha."""
    return PosteriorMeans.apply(context, Phi, y, alpha, em_iter)
