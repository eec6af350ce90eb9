"""torch.autograd wrappers: the SENSE NUFFT pair and the unrolled l2 PDHG, differentiable with
respect to the data, the l2 weight lambda and the trajectory coordinates.

Every forward and backward runs in libkpdhg's kernels (adjoint NUFFT, Kaiser-Bessel-derivative
gridding, the unrolled iteration's reverse sweep).  The plan must already hold the trajectory
passed as `traj` (set with Plan.set_trajectory); `traj` is taken as an autograd input only so
that its gradient can be returned.  Complex gradients follow PyTorch's convention
(dL/dRe + i dL/dIm).
"""
from __future__ import annotations

import torch


class SenseForward(torch.autograd.Function):
    """y = A x (Sec. 2, Eq. model_i, NUFFT approximation)."""

    @staticmethod
    def forward(ctx, x, traj, plan):
        ctx.plan = plan
        ctx.save_for_backward(x)
        return plan.sense_forward(x.contiguous())

    @staticmethod
    def backward(ctx, gy):
        (x,) = ctx.saved_tensors
        gy = gy.contiguous()
        gx = ctx.plan.sense_adjoint(gy) if ctx.needs_input_grad[0] else None
        gt = ctx.plan.sense_forward_traj_grad(x.contiguous(), gy) if ctx.needs_input_grad[1] else None
        return gx, gt, None


class SenseAdjoint(torch.autograd.Function):
    """x = A^H y."""

    @staticmethod
    def forward(ctx, y, traj, plan):
        ctx.plan = plan
        ctx.save_for_backward(y)
        return plan.sense_adjoint(y.contiguous())

    @staticmethod
    def backward(ctx, gx):
        (y,) = ctx.saved_tensors
        gx = gx.contiguous()
        gy = ctx.plan.sense_forward(gx) if ctx.needs_input_grad[0] else None
        gt = ctx.plan.sense_adjoint_traj_grad(y.contiguous(), gx) if ctx.needs_input_grad[1] else None
        return gy, gt, None


class UnrolledPDHG(torch.autograd.Function):
    """x_K of `iters` preconditioned PDHG iterations (Sec. 4.1) for g = lambda ||x||^2 / 2, with
    per-iteration checkpoints kept in the plan; p, lambda_max and the step sizes are constants."""

    @staticmethod
    def forward(ctx, y, lam, traj, plan, p, iters, lmax):
        ctx.plan = plan
        return plan.unrolled_forward(y.contiguous(), p, float(lam), int(iters), float(lmax))

    @staticmethod
    def backward(ctx, gx):
        gy, gl, gt = ctx.plan.unrolled_backward(gx.contiguous(), want_y=ctx.needs_input_grad[0],
                                                want_traj=ctx.needs_input_grad[2])
        glam = torch.tensor(gl, dtype=torch.float32, device=gx.device) if ctx.needs_input_grad[1] else None
        return gy, glam, gt, None, None, None, None


def sense_forward(x, traj, plan):
    return SenseForward.apply(x, traj, plan)


def sense_adjoint(y, traj, plan):
    return SenseAdjoint.apply(y, traj, plan)


def unrolled_pdhg(y, lam, traj, plan, p=None, iters=10, lmax=0.0):
    return UnrolledPDHG.apply(y, lam, traj, plan, p, iters, lmax)
