"""torch.autograd front of the library's log|psi| and its hand-written backward.

LogPsi.apply(params, occ, M0, context) returns log|psi(n_b)| for every configuration of the
batch. Its backward calls scale_grad_logpsi: the per-sample gradients
d log|psi_b| / d theta (Phi^-T pushed back through the projection, every layer and the
embedding, all in the CUDA library). They are kept on the autograd context as
`per_sample` [B][P] for a variational update, which needs the per-sample matrix and not only
the batch sum. Every step runs in the CUDA library; torch only holds memory and the graph.
"""
from __future__ import annotations

import torch

from .binding import Context


class LogPsi(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, occ: torch.Tensor, M0: torch.Tensor, context: Context,
                recompute: bool = False):
        if params.dtype != torch.float64 or not params.is_cuda:
            raise TypeError("params must be a float64 CUDA tensor")
        context.scale_set_params(params.detach().contiguous(), M0.contiguous())
        context.scale_load(occ.contiguous())
        la, _ = context.log_psi()
        ctx.context = context
        ctx.recompute = recompute
        return la

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        g = ctx.context.grad_logpsi(recompute=ctx.recompute)  # [B][P]
        ctx.per_sample = g
        return (grad_out.to(g.dtype)[:, None] * g).sum(0), None, None, None, None


def log_psi(params: torch.Tensor, occ: torch.Tensor, M0: torch.Tensor, context: Context,
            recompute: bool = False) -> torch.Tensor:
    return LogPsi.apply(params, occ, M0, context, recompute)


def per_sample_gradients(params: torch.Tensor, occ: torch.Tensor, M0: torch.Tensor,
                         context: Context, recompute: bool = False) -> torch.Tensor:
    """O[b][p] = d log|psi(n_b)| / d theta_p, computed by the library's backward kernels."""
    context.scale_set_params(params.detach().contiguous(), M0.contiguous())
    context.scale_load(occ.contiguous())
    return context.grad_logpsi(recompute=recompute)
