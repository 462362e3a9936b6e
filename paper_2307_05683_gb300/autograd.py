"""torch.autograd.Function around the library's adjoint.

    loss = final_position_loss(masses, pos, vel, n_planets, dt, target, n_steps)
    loss.sum().backward()     # fills masses.grad, pos.grad, vel.grad

loss[s] = sum_i |Q_i(T) - target[s, i]|^2 over the heliocentric positions of
the synchronized state after n_steps Wisdom-Holman steps.  forward runs the
checkpointed forward pass (whg_adjoint_forward), backward the adjoint kernels
(whg_adjoint_backward) with the incoming loss gradient as per-system weights.
All tensors live on the GPU in float64 (layouts of include/whg.h).
"""
from __future__ import annotations

import torch

from . import whg


class FinalPositionLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, masses, pos, vel, n_planets, dt, target, n_steps, checkpoint_every, gr_mode,
                lanes_per_system):
        S, B = masses.shape
        it = whg.Integrator(S, B - 1, gr_mode=gr_mode, lanes_per_system=lanes_per_system,
                            stream=torch.cuda.current_stream().cuda_stream)
        whg.whg_init_device(it.ctx, masses.contiguous(), pos.contiguous(), vel.contiguous(),
                            None if n_planets is None else n_planets.contiguous(), dt.contiguous())
        loss = torch.empty(S, dtype=torch.float64, device=masses.device)
        whg.whg_adjoint_forward(it.ctx, int(n_steps), int(checkpoint_every), target.contiguous(), loss)
        ctx.it = it
        ctx.shapes = (masses.shape, pos.shape)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        mshape, pshape = ctx.shapes
        dev = grad_loss.device
        gm = torch.empty(mshape, dtype=torch.float64, device=dev)
        gx = torch.empty(pshape, dtype=torch.float64, device=dev)
        gu = torch.empty(pshape, dtype=torch.float64, device=dev)
        whg.whg_adjoint_backward(ctx.it.ctx, grad_loss.contiguous().to(torch.float64), gx, gu, gm)
        ctx.it.synchronize()
        ctx.it.close()
        return gm, gx, gu, None, None, None, None, None, None, None


def final_position_loss(masses, pos, vel, n_planets, dt, target, n_steps, checkpoint_every=100,
                        gr_mode=1, lanes_per_system=0):
    return FinalPositionLoss.apply(masses, pos, vel, n_planets, dt, target, n_steps, checkpoint_every,
                                   gr_mode, lanes_per_system)
