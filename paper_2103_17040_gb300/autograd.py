"""PyTorch autograd wrapper of the discrete adjoint (argument marshalling only).

``mean_macro_concentration(params, problem, u0, v0, dt, nsteps)`` returns
J = int_Omega u(t_N) dx as a 0-d tensor whose gradient with respect to the
per-node deformation parameters comes from the library's hand-written
discrete adjoint (tsf_adjoint_mean_u: checkpointed forward march, backward
march with adjoint steps, gradient contraction on the GPU).  The adjoint runs
together with the forward march, so backward() only scales the stored
gradient.
"""
from __future__ import annotations

import numpy as np
import torch


class MeanMacroConcentration(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, problem, family, u0, v0, dt, nsteps, ckpt_every):
        problem.set_deformation(family, params.detach())
        problem.set_state(u0, v0)
        J, g = problem.adjoint_mean_u(dt, nsteps, ckpt_every)
        ctx.save_for_backward(torch.as_tensor(np.asarray(g), dtype=params.dtype, device=params.device)
                              .reshape(params.shape))
        return torch.tensor(J, dtype=params.dtype, device=params.device)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return gJ * g, None, None, None, None, None, None, None


def mean_macro_concentration(params, problem, family, u0, v0, dt, nsteps, ckpt_every=10):
    return MeanMacroConcentration.apply(params, problem, family, u0, v0, dt, nsteps, ckpt_every)
