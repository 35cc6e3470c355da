"""torch.autograd bridge: the moment series of a coil run as a differentiable
function of the calibration parameters (per-element Jc factor, n, C_eps).

forward runs the steps through the C ABI and returns the moment after every
step; backward calls coil_adjoint (hand-written reverse of the step with
checkpointed recomputation).  Tensors are CPU float64; the GPU work happens
inside the library.
"""
import numpy as np
import torch


class CoilMoments(torch.autograd.Function):
    """m = CoilMoments.apply(coil, drive, n_steps, ckpt_every, jc_factor, n, C_eps)."""

    @staticmethod
    def forward(ctx, coil, drive, n_steps, ckpt_every, jc_factor, n, C_eps):
        coil.set_params(jc_factor.detach().cpu().numpy(), float(n), float(C_eps))
        ctx.coil, ctx.drive, ctx.n_steps, ctx.ckpt = coil, drive, int(n_steps), int(ckpt_every)
        ctx.state0 = coil.save_state()
        first = coil.info().steps
        coil.step(n_steps, drive)
        m = coil.diag(first, n_steps)[:, 3].copy()
        return torch.from_numpy(m)

    @staticmethod
    def backward(ctx, grad_m):
        coil = ctx.coil
        after = coil.save_state()
        coil.load_state(ctx.state0)
        gf, gn, gc = coil.adjoint(ctx.n_steps, ctx.drive, grad_m.detach().cpu().numpy().astype(np.float64),
                                  ctx.ckpt)
        coil.load_state(after)
        return (None, None, None, None, torch.from_numpy(gf), torch.tensor(gn, dtype=torch.float64),
                torch.tensor(gc, dtype=torch.float64))
