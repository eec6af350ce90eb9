"""torch.autograd wrappers: the SENSE NUFFT pair and the unrolled l2 PDHG, differentiable with
respect to the data, the l2 weight lambda and the trajectory coordinates.

Every forward and backward runs in libkpdhg's kernels (adjoint NUFFT, Kaiser-Bessel-derivative
gridding, the unrolled iteration's reverse sweep).  The operator is the plan's: a `traj` whose
values differ from the plan's trajectory is set into the plan first (a new binning), so the
gradient is always that of the trajectory passed.  The unrolled solver's checkpoints live in the
plan, so only the plan's latest unrolled forward can be differentiated; backward through an
older one raises.  Complex gradients follow PyTorch's convention (dL/dRe + i dL/dIm).
"""
from __future__ import annotations

import torch


def _use_traj(plan, traj):
    """Make the plan's operator the one of `traj` (set it when its values differ)."""
    t = traj.detach()
    cur = getattr(plan, "trajectory", None)
    if cur is None or cur.shape != t.shape or not torch.equal(cur, t):
        plan.set_trajectory(t.contiguous())


class SenseForward(torch.autograd.Function):
    """y = A x (Sec. 2, Eq. model_i, NUFFT approximation)."""

    @staticmethod
    def forward(ctx, x, traj, plan):
        _use_traj(plan, traj)
        ctx.plan = plan
        ctx.traj = traj.detach()
        ctx.save_for_backward(x)
        return plan.sense_forward(x.contiguous())

    @staticmethod
    def backward(ctx, gy):
        (x,) = ctx.saved_tensors
        gy = gy.contiguous()
        _use_traj(ctx.plan, ctx.traj)
        gx = ctx.plan.sense_adjoint(gy) if ctx.needs_input_grad[0] else None
        gt = ctx.plan.sense_forward_traj_grad(x.contiguous(), gy) if ctx.needs_input_grad[1] else None
        return gx, gt, None


class SenseAdjoint(torch.autograd.Function):
    """x = A^H y."""

    @staticmethod
    def forward(ctx, y, traj, plan):
        _use_traj(plan, traj)
        ctx.plan = plan
        ctx.traj = traj.detach()
        ctx.save_for_backward(y)
        return plan.sense_adjoint(y.contiguous())

    @staticmethod
    def backward(ctx, gx):
        (y,) = ctx.saved_tensors
        gx = gx.contiguous()
        _use_traj(ctx.plan, ctx.traj)
        gy = ctx.plan.sense_forward(gx) if ctx.needs_input_grad[0] else None
        gt = ctx.plan.sense_adjoint_traj_grad(y.contiguous(), gx) if ctx.needs_input_grad[1] else None
        return gy, gt, None


class UnrolledPDHG(torch.autograd.Function):
    """x_K of `iters` preconditioned PDHG iterations (Sec. 4.1) for g = lambda ||x||^2 / 2, with
    per-iteration checkpoints kept in the plan; p, lambda_max and the step sizes are constants."""

    @staticmethod
    def forward(ctx, y, lam, traj, plan, p, iters, lmax):
        _use_traj(plan, traj)
        ctx.plan = plan
        x = plan.unrolled_forward(y.contiguous(), p, float(lam), int(iters), float(lmax))
        ctx.tape_id = plan.tape_id
        return x

    @staticmethod
    def backward(ctx, gx):
        if getattr(ctx.plan, "tape_id", None) != ctx.tape_id:
            raise RuntimeError("the plan's checkpoints belong to a later unrolled forward; run the unrolled "
                               "forward again (or use one plan per graph) before differentiating this one")
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
