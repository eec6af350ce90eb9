"""GPU parity of the l2-optimised diagonal k-space preconditioners (Sec. 5, Eq. sc_precond /
mc_precond, fast route of Sec. 5.1) against the float64 oracle's fast route at the same NUFFT
settings, plus the Cartesian pin (p = 1, Sec. 5) on the GPU.

Tolerance 1e-5 relative l2 (the float32-operator bar).  The GPU route runs its FFTs and
gridding in float32 and accumulates the denominator sums (R_c over coil pairs, the taps of the
final type-2 interpolation) in float64; emulating every float32 step of the route on the CPU
gives about 1e-7 on these cases."""
import numpy as np
import pytest

from oracle import precond as opc
from tests.gpu_util import need_gpu, rel, random_problem, workload_problem, to_dev, make_plan

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,C,M,seed", [((24, 20), 3, 400, 1), ((12, 16, 8), 2, 300, 2), ((40, 36), 5, 3000, 3)])
def test_mc_sc_random(shape, C, M, seed):
    need_gpu()
    _, maps, traj = random_problem(shape, C, M, seed, edge=True)
    maps = maps / np.sqrt(np.sum(np.abs(maps) ** 2, axis=0, keepdims=True))
    p_mc = opc.mc_precond_fast(maps.astype(np.complex128), traj, 1.25, 4)
    p_sc = opc.sc_precond_fast(traj, shape, 1.25, 4)
    plan = make_plan(shape, C, M)
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    g_mc = plan.make_preconditioner(True).cpu().numpy()
    g_sc = plan.make_preconditioner(False).cpu().numpy()
    assert rel(g_mc, p_mc, "mc") < 1e-5
    for c in range(C):
        assert rel(g_sc[c], p_sc, "sc") < 1e-5


def test_cartesian_single_channel_is_one():
    need_gpu()
    ky, kx = np.meshgrid(np.arange(-16, 16), np.arange(-12, 12), indexing="ij")
    traj = np.stack([ky.ravel(), kx.ravel()], -1).astype(np.float32)
    plan = make_plan((32, 24), 1, traj.shape[0], 2.0)
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(np.ones((1, 32, 24), np.complex64)))
    p = plan.make_preconditioner(False).cpu().numpy()
    # the paper's value 1, up to the alpha-2, W-4 interpolation error of the route's NUFFTs
    assert np.abs(p - 1).max() < 2e-2
    # and the oracle's fast route with the same NUFFT settings, to float32 rounding
    assert rel(p[0], opc.sc_precond_fast(traj, (32, 24), 2.0, 4), "cartesian") < 1e-5


@pytest.mark.parametrize("name,alpha", [("radial2d_128", 2.0), ("spiral2d_256", 1.25)])
def test_mc_workloads(name, alpha):
    need_gpu()
    w, x, maps, traj = workload_problem(name)
    p_ref = opc.mc_precond_fast(maps.astype(np.complex128), traj, alpha, 4)
    plan = make_plan(x.shape, maps.shape[0], traj.shape[0], alpha)
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    p = plan.make_preconditioner(True).cpu().numpy()
    assert (p > 0).all()
    assert rel(p, p_ref, name) < 1e-5
