"""torch.autograd.Function over the library's log-likelihood and its hand-written backward kernel.

The gradient of the multinomial-logit log-likelihood (Eq. 1; the paper prints no gradient) is
d ll_p / d theta_{p,c} = sum_{s<=t} (1[y_s = c] - p_{s,c}(theta_p)) x_s, computed by the
library's gradient kernel (sps_loglik_grad). Particles are independent, so the backward pass of
ll = loglik(theta) is grad_theta[p] = grad_ll[p] * G[p]. This module only marshals arguments:
both directions run in libsps.so kernels on torch's current stream.
"""
from __future__ import annotations

from typing import Optional

import torch


class LogLik(torch.autograd.Function):
    """ll [P] = log-likelihood of each row of theta [P, D] (CUDA, float64) over the first t
    observations; backward through the library's gradient kernel."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, sps, t: Optional[int], precision: str):
        ctx.sps = sps
        ctx.t = sps.n if t is None else int(t)
        ctx.save_for_backward(theta)
        return sps.loglik(theta.detach(), ctx.t, precision)

    @staticmethod
    def backward(ctx, grad_ll: torch.Tensor):
        (theta,) = ctx.saved_tensors
        _, g = ctx.sps.loglik_grad(theta.detach(), ctx.t)
        return grad_ll.to(g.dtype)[:, None] * g, None, None, None


def loglik(theta: torch.Tensor, sps, t: Optional[int] = None, precision: str = "split") -> torch.Tensor:
    """Differentiable log-likelihood of the particles theta [P, D] (see LogLik)."""
    return LogLik.apply(theta, sps, t, precision)
