"""torch.autograd.Function over the library's fitness and adjoint kernels.

``TGPFitness.apply(val, X, type_, size, y, n_outputs)`` returns the MSE
``[pop, n_outputs]`` (float64) of the population whose node values are
``val``; its backward calls ``tgp_eval_backward`` and returns the gradient with
respect to ``val`` (non-zero at constant nodes only) and to ``X``.  The
forward and backward both run in the CUDA library; this module only wires
them into autograd.
"""
from __future__ import annotations

import torch

from . import api


class TGPFitness(torch.autograd.Function):
    @staticmethod
    def forward(ctx, val, X, type_, size, y, n_outputs=1, max_len=None):
        mse, status = api.tgp_fitness_mse(type_, val.detach(), size, X.detach(), y, n_outputs,
                                          max_len=max_len)
        ctx.save_for_backward(val, X, type_, size, y)
        ctx.n_outputs = n_outputs
        ctx.max_len = max_len
        ctx.mark_non_differentiable(status)
        return mse, status

    @staticmethod
    def backward(ctx, grad_mse, grad_status):
        val, X, type_, size, y = ctx.saved_tensors
        need_v, need_x = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_v or need_x) or grad_mse is None:
            return (None,) * 7
        _, gv, gx, _ = api.tgp_eval_backward(type_, val.detach(), size, X.detach(), y, grad_mse,
                                             ctx.n_outputs, max_len=ctx.max_len, want_mse=False,
                                             want_grad_value=need_v, want_grad_X=need_x)
        return gv, gx, None, None, None, None, None


def fitness(val, X, type_, size, y, n_outputs=1, max_len=None):
    """MSE [pop, n_outputs] differentiable with respect to val and X."""
    mse, _ = TGPFitness.apply(val, X, type_, size, y, n_outputs, max_len)
    return mse
