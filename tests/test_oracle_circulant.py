"""Pins of the oracle's l2-optimised circulant preconditioner (App. B), its preconditioned CG and
the generic FISTA (the comparison systems of Sec. 6), without a GPU.

* the r/h route equals the argmin computed from a dense A^H A (2D and 3D);
* the argmin's normal equations: every circulant diagonal of A^H A - P sums to zero, and the
  objective grows by exactly N ||delta||^2 for any circulant perturbation delta (a quadratic
  with an exact minimiser);
* fully sampled Cartesian k-space with one unit coil: A^H A = I, so P = I (kernel = delta);
* Hermitian A^H A gives a Hermitian positive semidefinite P (real, non-negative eigenvalues);
* preconditioned CG and FISTA reach the l2 optimum that plain CG reaches.
"""
import numpy as np
import pytest

import synth
from oracle import nufft as nf
from oracle import precond as pc
from oracle import solvers as sv


def _tiny(shape, C, M, seed):
    rng = np.random.default_rng(seed)
    maps = rng.standard_normal((C,) + shape) + 1j * rng.standard_normal((C,) + shape)
    traj = np.stack([rng.uniform(-n / 2, n / 2, M) for n in shape], -1)
    return maps, traj


@pytest.mark.parametrize("shape,C,M,seed", [((6, 8), 2, 40, 1), ((4, 6, 4), 2, 30, 2)])
def test_route_equals_dense_argmin(shape, C, M, seed):
    maps, traj = _tiny(shape, C, M, seed)
    A = nf.sense_matrix(maps, traj)
    c_dense = pc.circulant_kernel_bruteforce(A, shape)
    c_route = pc.circulant_kernel(maps, traj, exact=True)
    assert np.abs(c_route - c_dense).max() < 1e-12 * np.abs(c_dense).max()


def test_normal_equations_and_exact_quadratic():
    shape, C, M = (6, 6), 2, 36
    maps, traj = _tiny(shape, C, M, 3)
    A = nf.sense_matrix(maps, traj)
    N = int(np.prod(shape))
    c = pc.circulant_kernel_bruteforce(A, shape)
    H = A.conj().T @ A
    idx = np.stack(np.unravel_index(np.arange(N), shape), -1)
    lag = np.mod(idx[:, None, :] - idx[None, :, :], np.array(shape))
    P = c[lag[..., 0], lag[..., 1]]
    diag_sums = np.zeros(shape, dtype=np.complex128)
    np.add.at(diag_sums, (lag[..., 0].ravel(), lag[..., 1].ravel()), (H - P).ravel())
    assert np.abs(diag_sums).max() < 1e-12 * np.abs(H).max() * N
    f0 = pc.circulant_objective(c, A, shape)
    rng = np.random.default_rng(4)
    delta = 1e-2 * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    f1 = pc.circulant_objective(c + delta, A, shape)
    assert abs((f1 - f0) - N * np.sum(np.abs(delta) ** 2)) < 1e-9 * f0


def test_cartesian_unit_coil_gives_identity():
    shape = (8, 6)
    ky, kx = np.meshgrid(np.arange(-4, 4), np.arange(-3, 3), indexing="ij")
    traj = np.stack([ky.ravel(), kx.ravel()], -1).astype(np.float64)
    c = pc.circulant_kernel(np.ones((1,) + shape), traj, exact=True)
    delta = np.zeros(shape)
    delta[0, 0] = 1.0
    assert np.abs(c - delta).max() < 1e-12


def test_hermitian_psd():
    shape, C, M = (8, 8), 3, 50
    maps, traj = _tiny(shape, C, M, 5)
    c = pc.circulant_kernel(maps, traj, exact=True)
    mirror = np.conj(c[np.ix_(*[np.mod(-np.arange(n), n) for n in shape])])
    assert np.abs(c - mirror).max() < 1e-12 * np.abs(c).max()
    ev = pc.circulant_eigenvalues(c)
    assert np.abs(ev.imag).max() < 1e-10 * np.abs(ev.real).max()
    assert ev.real.min() > -1e-10 * ev.real.max()


def test_pcg_and_fista_reach_the_l2_optimum():
    shape, C = (16, 16), 3
    maps = synth.coil_maps(shape, C, seed=2).astype(np.complex128)
    traj = synth.spiral_archimedean(6, 96, 8.0)
    A = lambda v: nf.nufft_forward(v, maps, traj, 1.25, 4)
    AH = lambda u: nf.nufft_adjoint(u, maps, traj, 1.25, 4)
    x0 = synth.ellipse_phantom(shape, seed=2).astype(np.complex128)
    y = A(x0) + 0.01 * synth.complex_noise((C, traj.shape[0]), 3)
    lam = 1e-2
    xs = sv.cg_l2(A, AH, y, lam, shape)
    ev = pc.circulant_eigenvalues(pc.circulant_kernel(maps, traj, 1.25, 4))
    x_pcg, objs = sv.pcg_l2_circulant(A, AH, y, lam, shape, ev, 240, trace=True)
    assert np.linalg.norm(x_pcg - xs) < 1e-9 * np.linalg.norm(xs)
    x_cg, objs_cg = sv.pcg_l2_circulant(A, AH, y, lam, shape, None, 240, trace=True)
    assert np.linalg.norm(x_cg - xs) < 1e-7 * np.linalg.norm(xs)
    # on this variable-density spiral the circulant preconditioner speeds CG up per iteration
    assert objs[119] < objs_cg[119]
    L, _ = sv.power_method(A, AH, 1.0, shape, iters=100)
    x_f, fo = sv.fista(A, AH, y, "l2", lam, shape, 1.0001 * L, 2000, trace=True)
    Fs = sv.objective(A, xs, y, "l2", lam)
    # FISTA's objective gap falls like 1/k^2 (here 6e-4 at 100 and 6e-9 at 2000 iterations)
    assert (fo[-1] - Fs) < 2e-8 * Fs and (fo[99] - Fs) > 100 * (fo[-1] - Fs)
    assert np.linalg.norm(x_f - xs) < 2e-4 * np.linalg.norm(xs)
    assert min(objs) >= Fs * (1 - 1e-12) and min(fo) >= Fs * (1 - 1e-12)
