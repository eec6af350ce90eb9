"""GPU parity of the l2-optimised diagonal k-space preconditioners (Sec. 5, Eq. sc_precond /
mc_precond, fast route of Sec. 5.1) against the oracle's fast route at the same NUFFT
settings, plus the Cartesian pin (p = 1, Sec. 5) on the GPU.

Tolerance 1e-4 relative l2: the route's float32 FFT of |Q_cd|^2 and the final float32
type-2 NUFFT each carry ~1e-6 relative error of the largest term, and the denominator is a
sum of positive terms whose small entries (edge of k-space) amplify that by up to ~1e2."""
import numpy as np
import pytest

from oracle import precond as opc
from tests.gpu_util import need_gpu, rel, random_problem, workload_problem, to_dev, make_plan

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,C,M,seed", [((24, 20), 3, 400, 1), ((12, 16, 8), 2, 300, 2)])
def test_mc_sc_random(shape, C, M, seed):
    need_gpu()
    _, maps, traj = random_problem(shape, C, M, seed)
    maps = maps / np.sqrt(np.sum(np.abs(maps) ** 2, axis=0, keepdims=True))
    p_mc = opc.mc_precond_fast(maps.astype(np.complex128), traj, 1.25, 4)
    p_sc = opc.sc_precond_fast(traj, shape, 1.25, 4)
    plan = make_plan(shape, C, M)
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    g_mc = plan.make_preconditioner(True).cpu().numpy()
    g_sc = plan.make_preconditioner(False).cpu().numpy()
    assert rel(g_mc, p_mc) < 1e-4
    for c in range(C):
        assert rel(g_sc[c], p_sc) < 1e-4


def test_cartesian_single_channel_is_one():
    need_gpu()
    ky, kx = np.meshgrid(np.arange(-16, 16), np.arange(-12, 12), indexing="ij")
    traj = np.stack([ky.ravel(), kx.ravel()], -1).astype(np.float32)
    plan = make_plan((32, 24), 1, traj.shape[0], 2.0)
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(np.ones((1, 32, 24), np.complex64)))
    p = plan.make_preconditioner(False).cpu().numpy()
    # NUFFT-approximated route: 1 up to the alpha-2, W-4 interpolation error
    assert np.abs(p - 1).max() < 2e-2


@pytest.mark.parametrize("name,alpha", [("radial2d_128", 2.0), ("spiral2d_256", 1.25)])
def test_mc_workloads(name, alpha):
    need_gpu()
    w, x, maps, traj = workload_problem(name)
    p_ref = opc.mc_precond_fast(maps.astype(np.complex128), traj, alpha, 4)
    plan = make_plan(x.shape, maps.shape[0], traj.shape[0], alpha)
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    p = plan.make_preconditioner(True).cpu().numpy()
    assert (p > 0).all()
    assert rel(p, p_ref) < 1e-4
