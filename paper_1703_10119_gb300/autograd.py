"""The misfit loss of a batch of walls as a differentiable function of the layer parameters.

``MisfitLoss.apply(theta, ctx, n_steps, sample_every, obs, wT, wP)`` returns the sensor-misfit loss of a
run of the walls held by ``ctx`` (a :class:`~paper_1703_10119_gb300.hygro.Hygro`) with the per-layer
parameters ``theta`` ([total layers, 9]: kM0, a, cM0, b, kTT0, aT, cTT0, bT, chi), and its backward hands
back the gradient that ``hygro_loss_grad`` computes with the reverse-time adjoint on the GPU. Argument
marshalling only: the forward run, the loss and the gradient come from the CUDA library.

Side effect on ``ctx``: its materials become ``theta`` (``hygro_set_materials``, which also resets the
stored levels to the initial state). The context's run state (both stored levels, the step, the flux
sums and the room air) is saved before and restored after, so a run of ``ctx`` that was under way goes
on from where it was, now with the materials ``theta``.
"""
from __future__ import annotations

import numpy as np
import torch


class MisfitLoss(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, ctx, n_steps: int, sample_every: int, obs, wT: float, wP: float,
                checkpoint_every: int = 0):
        par = theta.detach().to("cpu", torch.float64).numpy()
        saved = ctx.get_state()
        ctx.set_materials(par)
        try:
            loss, grad = ctx.loss_grad(n_steps, sample_every, obs, wT, wP, checkpoint_every)
        finally:
            ctx.set_state(saved)
        fctx.save_for_backward(torch.from_numpy(np.ascontiguousarray(grad)).to(theta.device, theta.dtype))
        return torch.tensor(loss, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(fctx, grad_out):
        (g,) = fctx.saved_tensors
        return grad_out * g, None, None, None, None, None, None, None
