"""GPU parity of the l2 reconstruction through the dual (appendix on the connection to Trzasko
et al.): (A A^H + lambda I) w = lambda y by conjugate gradients with the diagonal k-space
preconditioner p (or none), x = A^H w / lambda, through kp_dual_l2_solve, against the float64
oracle's dual_l2_pcg on the same inputs.  Tolerance 1e-5 relative on x and on every entry of
the residual trace (relative to the first residual ||lambda y||).

Without P the system A A^H + lambda I is badly conditioned here and conjugate gradients amplify
rounding: on the CPU, the same recursion with its vectors rounded to complex64 departs from
float64 by 4e-8 after 5 iterations, 1.4e-5 after 8 and 0.2 after 15.  That case is compared
over 5 iterations; with P (20 iterations) float32 and float64 agree to 4e-7.  Both routes reach
the primal optimum when run to convergence (last test)."""
import numpy as np
import pytest

import synth
from oracle import nufft as onf, precond as opc, solvers as osv
from tests.gpu_util import need_gpu, rel, simulate, to_dev, make_plan

pytestmark = pytest.mark.gpu


def _problem(n=48, C=3, L=6, ns=768):
    w = synth.Workload("dual_small", (n, n), C, 1.25, 4, "l2", 1e-2, 20, 0, "spiral",
                       dict(n_interleaves=L, n_samples=ns, kmax=n / 2.0))
    x, maps, traj = w.phantom(), w.maps(), w.traj()
    return w, x, maps, traj, simulate(w, x, maps, traj)


@pytest.mark.parametrize("use_p,iters", [(True, 20), (False, 5)])
def test_dual_l2_matches_oracle(use_p, iters):
    need_gpu()
    w, x, maps, traj, y = _problem()
    m = maps.astype(np.complex128)
    A = lambda v: onf.nufft_forward(v, m, traj, 1.25, 4)
    AH = lambda u: onf.nufft_adjoint(u, m, traj, 1.25, 4)
    p = opc.mc_precond_fast(m, traj, 1.25, 4) if use_p else np.ones(y.shape)
    lam = 0.05
    x_ref, w_ref, res_ref = osv.dual_l2_pcg(A, AH, y, p, lam, iters)
    plan = make_plan(x.shape, maps.shape[0], traj.shape[0])
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    pd = to_dev(p.astype(np.float32)) if use_p else None
    xg, res = plan.dual_l2_solve(to_dev(y), pd, lam, iters)
    assert rel(xg.cpu().numpy(), x_ref, "x") < 1e-5
    res, res_ref = np.array(res), np.array(res_ref)
    assert np.abs(res - res_ref).max() < 1e-5 * res_ref[0]
    if use_p:
        assert res[-1] < 0.1 * res[0]
    # a second call on the same plan (buffers reused) repeats the result up to the order of the
    # float atomics of split spreading tiles
    xg2, _ = plan.dual_l2_solve(to_dev(y), pd, lam, iters)
    assert rel(xg2.cpu().numpy(), xg.cpu().numpy(), "repeat") < 1e-5


def test_dual_l2_reaches_primal_optimum():
    """Run to convergence, the dual route gives the primal ridge solution (A^H A + lambda I)^{-1}
    A^H y of Eq. obj with g = lambda ||x||^2 / 2 (oracle CG on the normal equations)."""
    need_gpu()
    w, x, maps, traj, y = _problem(n=32, C=2, L=4, ns=512)
    m = maps.astype(np.complex128)
    A = lambda v: onf.nufft_forward(v, m, traj, 1.25, 4)
    AH = lambda u: onf.nufft_adjoint(u, m, traj, 1.25, 4)
    lam = 0.05
    xs = osv.cg_l2(A, AH, y, lam, x.shape)
    plan = make_plan(x.shape, maps.shape[0], traj.shape[0])
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    xg, res = plan.dual_l2_solve(to_dev(y), None, lam, 150)
    assert res[-1] < 1e-4 * res[0]
    assert rel(xg.cpu().numpy(), xs, "x vs primal optimum") < 1e-4


def test_dual_l2_rejects_bad_inputs():
    need_gpu()
    from paper_1902_09657_gb300._lib import KpError
    w, x, maps, traj, y = _problem(n=32, C=2, L=4, ns=512)
    plan = make_plan(x.shape, maps.shape[0], traj.shape[0])
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    with pytest.raises(KpError):
        plan.dual_l2_solve(to_dev(y), None, 0.0, 5)
    bad = np.ones(y.shape, np.float32)
    bad[1, 7] = -1.0
    with pytest.raises(KpError):
        plan.dual_l2_solve(to_dev(y), to_dev(bad), 0.05, 5)
