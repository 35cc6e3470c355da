"""torch.autograd bridge: the per-step series of a coil run as differentiable
functions of the calibration parameters (per-element Jc factor, n, C_eps).

CoilMoments: the moment after every step (a magnetization-loop loss).
CoilSeries: the moment after every step and the Joule power of every step's
start state (a magnetization-loop loss plus, e.g., a soft maximum of the
Joule power as a smooth quench-onset loss).

forward runs the steps through the C ABI and returns the series; backward
calls the hand-written reverse of the step with checkpointed recomputation
(coil_adjoint / coil_adjoint_losses).  Tensors are CPU float64; the GPU work
happens inside the library.
"""
import numpy as np
import torch


def _run(ctx, coil, drive, n_steps, ckpt_every, jc_factor, n, C_eps):
    coil.set_params(jc_factor.detach().cpu().numpy(), float(n), float(C_eps))
    ctx.coil, ctx.drive, ctx.n_steps, ctx.ckpt = coil, drive, int(n_steps), int(ckpt_every)
    ctx.state0 = coil.save_state()
    first = coil.info().steps
    coil.step(n_steps, drive)
    return coil.diag(first, n_steps)


def _grads(gf, gn, gc):
    return torch.from_numpy(gf), torch.tensor(gn, dtype=torch.float64), torch.tensor(gc, dtype=torch.float64)


class CoilMoments(torch.autograd.Function):
    """m = CoilMoments.apply(coil, drive, n_steps, ckpt_every, jc_factor, n, C_eps)."""

    @staticmethod
    def forward(ctx, coil, drive, n_steps, ckpt_every, jc_factor, n, C_eps):
        d = _run(ctx, coil, drive, n_steps, ckpt_every, jc_factor, n, C_eps)
        return torch.from_numpy(d[:, 3].copy())

    @staticmethod
    def backward(ctx, grad_m):
        coil = ctx.coil
        after = coil.save_state()
        coil.load_state(ctx.state0)
        gf, gn, gc = coil.adjoint(ctx.n_steps, ctx.drive, grad_m.detach().cpu().numpy().astype(np.float64),
                                  ctx.ckpt)
        coil.load_state(after)
        return (None, None, None, None) + _grads(gf, gn, gc)


class CoilSeries(torch.autograd.Function):
    """(m, P) = CoilSeries.apply(coil, drive, n_steps, ckpt_every, jc_factor, n, C_eps):
    the moment after every step and the Joule power of every step's start state."""

    @staticmethod
    def forward(ctx, coil, drive, n_steps, ckpt_every, jc_factor, n, C_eps):
        d = _run(ctx, coil, drive, n_steps, ckpt_every, jc_factor, n, C_eps)
        return torch.from_numpy(d[:, 3].copy()), torch.from_numpy(d[:, 4].copy())

    @staticmethod
    def backward(ctx, grad_m, grad_P):
        coil = ctx.coil
        after = coil.save_state()
        coil.load_state(ctx.state0)
        gm = None if grad_m is None else grad_m.detach().cpu().numpy().astype(np.float64)
        gp = None if grad_P is None else grad_P.detach().cpu().numpy().astype(np.float64)
        if gm is None and gp is None:
            gm = np.zeros(ctx.n_steps)
        gf, gn, gc = coil.adjoint_losses(ctx.n_steps, ctx.drive, gm, gp, ctx.ckpt)
        coil.load_state(after)
        return (None, None, None, None) + _grads(gf, gn, gc)
