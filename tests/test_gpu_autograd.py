"""GPU parity of the differentiable pieces against the float64 oracle (trajectory gradients
of the SENSE pair; gradients of the unrolled l2 PDHG w.r.t. y, lambda and the trajectory),
through the C ABI and the torch.autograd wrappers.

Tolerances: 1e-5 relative l2 for x and the y-gradients, 1e-4 for lambda and the trajectory
gradients, which sum Kaiser-Bessel derivative terms of both signs over the window (the
cancellation amplifies float32 rounding)."""
import numpy as np
import pytest

import synth
from oracle import gradients as og
from oracle import nufft as onf, precond as opc, solvers as osv
from tests.gpu_util import need_gpu, rel, random_problem, to_dev, make_plan, simulate, workload_problem

pytestmark = pytest.mark.gpu


def test_sense_traj_gradients():
    need_gpu()
    import torch
    x, maps, traj = random_problem((32, 24), 3, 600, 21)
    rng = np.random.default_rng(22)
    gy = (rng.standard_normal((3, 600)) + 1j * rng.standard_normal((3, 600))).astype(np.complex64)
    gx = (rng.standard_normal((32, 24)) + 1j * rng.standard_normal((32, 24))).astype(np.complex64)
    ref_f = og.traj_grad_forward(x.astype(np.complex128), maps.astype(np.complex128), traj, gy.astype(np.complex128))
    ref_a = og.traj_grad_adjoint(gy.astype(np.complex128), maps.astype(np.complex128), traj, gx.astype(np.complex128))
    plan = make_plan((32, 24), 3, 600)
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    gf = plan.sense_forward_traj_grad(to_dev(x), to_dev(gy)).cpu().numpy()
    ga = plan.sense_adjoint_traj_grad(to_dev(gy), to_dev(gx)).cpu().numpy()
    assert rel(gf, ref_f, "forward traj grad") < 1e-4
    assert rel(ga, ref_a, "adjoint traj grad") < 1e-4
    # through torch.autograd
    from paper_1902_09657_gb300.autograd import sense_forward, sense_adjoint
    xt = to_dev(x).requires_grad_(True)
    tt = to_dev(traj).requires_grad_(True)
    y = sense_forward(xt, tt, plan)
    (y.conj() * to_dev(gy)).real.sum().backward()
    assert rel(tt.grad.cpu().numpy(), ref_f, "autograd traj grad") < 1e-4
    ref_gx = onf.nufft_adjoint(gy.astype(np.complex128), maps.astype(np.complex128), traj)
    assert rel(xt.grad.cpu().numpy(), ref_gx) < 1e-5


def _unrolled_problem(n=32, C=2, L=6, ns=512):
    w = synth.Workload("unrolled_small", (n, n), C, 1.25, 4, "l2", 1e-2, 10, 0, "spiral",
                       dict(n_interleaves=L, n_samples=ns, kmax=n / 2.0))
    return w, w.phantom(), w.maps(), w.traj()


def test_unrolled_gradients_match_oracle():
    need_gpu()
    import torch
    w, x, maps, traj = _unrolled_problem()
    y = simulate(w, x, maps, traj)
    m = maps.astype(np.complex128)
    A = lambda v: onf.nufft_forward(v, m, traj)
    AH = lambda u: onf.nufft_adjoint(u, m, traj)
    p = opc.mc_precond_fast(m, traj, 1.25, 4)
    Lmax, _ = osv.power_method(A, AH, p, x.shape, iters=30)
    lam, K = 1e-2, 10
    rng = np.random.default_rng(5)
    c = (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)).astype(np.complex64)
    xK, tape = og.unrolled_pdhg_l2(y, m, traj, p, lam, K, Lmax)
    gy_ref, gl_ref, gt_ref = og.unrolled_pdhg_l2_grad(c.astype(np.complex128), y, m, traj, p, lam, K, Lmax, tape)
    plan = make_plan(x.shape, maps.shape[0], traj.shape[0])
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    from paper_1902_09657_gb300.autograd import unrolled_pdhg
    yt = to_dev(y).requires_grad_(True)
    lt = torch.tensor(lam, dtype=torch.float32, device="cuda", requires_grad=True)
    tt = to_dev(traj).requires_grad_(True)
    xg = unrolled_pdhg(yt, lt, tt, plan, to_dev(p.astype(np.float32)), K, Lmax)
    assert rel(xg.detach().cpu().numpy(), xK) < 1e-5
    (xg.conj() * to_dev(c)).real.sum().backward()
    assert rel(yt.grad.cpu().numpy(), gy_ref, "dL/dy") < 1e-5
    assert abs(float(lt.grad) - gl_ref) < 1e-4 * abs(gl_ref)
    assert rel(tt.grad.cpu().numpy(), gt_ref, "dL/dtraj") < 1e-4


def test_unrolled_full_size_adjointness():
    """Differentiable workload at full size (256^2, 16 coils, 16 x 4096 spiral, 10 iterations):
    the y -> x_K map is linear, so <g_y, dy> must equal <c, x_K(dy)>, both from the GPU."""
    need_gpu()
    import torch
    w, x, maps, traj = workload_problem("spiral2d_256_unrolled")
    C, M = maps.shape[0], traj.shape[0]
    plan = make_plan(x.shape, C, M)
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    p = plan.make_preconditioner(True)
    Lmax = plan.max_eig(p)
    g = torch.Generator(device="cuda").manual_seed(1)
    y = plan.sense_forward(to_dev(x))
    c = torch.randn(x.shape, dtype=torch.complex64, device="cuda", generator=g)
    dy = torch.randn((C, M), dtype=torch.complex64, device="cuda", generator=g)
    plan.unrolled_forward(y, p, 1e-2, 10, Lmax)
    gy, gl, gt = plan.unrolled_backward(c)
    xd = plan.unrolled_forward(dy, p, 1e-2, 10, Lmax)
    lhs = float(torch.vdot(gy.flatten().to(torch.complex128), dy.flatten().to(torch.complex128)).real)
    rhs = float(torch.vdot(c.flatten().to(torch.complex128), xd.flatten().to(torch.complex128)).real)
    assert abs(lhs - rhs) < 1e-4 * abs(rhs)
    assert np.isfinite(gl) and bool(torch.isfinite(gt).all())
