"""The plateau-reduced loss as a torch.autograd.Function.

forward(theta) runs one plateau-reduced gradient estimate on the GPU (Eq. 10: the R
perturbed renders, their image losses and the kernel-weighted difference) and returns
the mean of the R perturbed losses -- the monitored loss; with importance-sampled
perturbations it is not an unbiased estimate of the smoothed objective, which is why
the gradient is not obtained by differentiating it. backward() returns the saved
estimator output times the incoming gradient: the estimator *is* the backward pass.

Each forward call advances the Philox step counter of its options object, so
consecutive calls draw fresh perturbations.
"""
from __future__ import annotations

import torch

from . import api


class SmoothedLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, scene: api.Scene, sigma: torch.Tensor, target: torch.Tensor, opts):
        theta_c = theta.detach().to(torch.float32).contiguous()
        grad, losses = scene.smoothed_grad(theta_c, sigma, target, opts)
        ctx.save_for_backward(grad)
        ctx.theta_dtype = theta.dtype
        return losses.mean()

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return (grad_out * grad).to(ctx.theta_dtype), None, None, None, None


class PlateauReducedLoss(torch.nn.Module):
    """Module wrapper: loss = PlateauReducedLoss(scene, wl, target)(theta); loss.backward()."""

    def __init__(self, scene: api.Scene, wl, target: torch.Tensor, sigma: torch.Tensor | None = None, step0: int = 0):
        super().__init__()
        self.scene = scene
        self.wl = wl
        self.target = target
        self.sigma = sigma if sigma is not None else torch.as_tensor(wl.sigma, device=target.device)
        self.step = step0

    def forward(self, theta: torch.Tensor) -> torch.Tensor:
        opts = self.scene.grad_opts(self.wl, step=self.step)
        self.step += 1
        return SmoothedLoss.apply(theta, self.scene, self.sigma, self.target, opts)
