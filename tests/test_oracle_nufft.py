"""Pins of the oracle's forward model and NUFFT (no GPU).

Exact model: Sec. 2, Eq. model_i (d-dimensional, centred index).  NUFFT: Sec. 6
(Kaiser-Bessel gridding following Beatty et al.).
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import nufft as nf


def _rand_problem(shape, C, M, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    maps = rng.standard_normal((C,) + shape) + 1j * rng.standard_normal((C,) + shape)
    traj = np.stack([rng.uniform(-n / 2, n / 2, M) for n in shape], -1).astype(np.float32)
    return x, maps, traj


def test_nudft_cartesian_equals_fft():
    """On a full Cartesian grid the exact model is a centred DFT (numpy.fft)."""
    shape = (8, 6)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    maps = np.ones((1,) + shape)
    ky, kx = np.meshgrid(np.arange(-4, 4), np.arange(-3, 3), indexing="ij")
    traj = np.stack([ky.ravel(), kx.ravel()], -1).astype(np.float32)
    y = nf.nudft_forward(x, maps, traj)[0]
    X = np.fft.fftn(np.fft.ifftshift(x)) / math.sqrt(x.size)
    ref = X[np.mod(ky.ravel(), 8), np.mod(kx.ravel(), 6)]
    assert np.abs(y - ref).max() < 1e-12


def test_dense_matrix_matches_samplewise_model():
    x, maps, traj = _rand_problem((6, 5), 2, 17, 1)
    A = nf.sense_matrix(maps, traj)
    y = nf.nudft_forward(x, maps, traj)
    assert np.abs(A @ x.ravel() - y.ravel()).max() < 1e-12
    u = np.random.default_rng(2).standard_normal((2, 17)) + 0j
    assert np.abs(A.conj().T @ u.ravel() - nf.nudft_adjoint(u, maps, traj).ravel()).max() < 1e-12


def test_nufft_converges_to_nudft_with_width():
    """NUFFT error falls with the kernel width and reaches < 1e-9 at W = 12, alpha = 2."""
    x, maps, traj = _rand_problem((16, 12), 3, 60, 3)
    ye = nf.nudft_forward(x, maps, traj)
    errs = []
    for W in (4, 6, 8, 12):
        y = nf.nufft_forward(x, maps, traj, 2.0, W)
        errs.append(np.linalg.norm(y - ye) / np.linalg.norm(ye))
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-9
    # the paper's setting (alpha 1.25, W 4) is a few-1e-3 approximation
    e = np.linalg.norm(nf.nufft_forward(x, maps, traj, 1.25, 4) - ye) / np.linalg.norm(ye)
    assert e < 2e-2


def test_nufft_3d_converges_to_nudft():
    x, maps, traj = _rand_problem((8, 6, 6), 2, 30, 4)
    ye = nf.nudft_forward(x, maps, traj)
    y = nf.nufft_forward(x, maps, traj, 2.0, 10)
    assert np.linalg.norm(y - ye) / np.linalg.norm(ye) < 1e-7


@pytest.mark.parametrize("alpha,W", [(1.25, 4), (2.0, 4), (2.0, 6)])
def test_adjoint_identity(alpha, W):
    x, maps, traj = _rand_problem((12, 10), 3, 40, 5)
    u = np.random.default_rng(6).standard_normal((3, 40)) + 1j * np.random.default_rng(7).standard_normal((3, 40))
    lhs = np.vdot(u, nf.nufft_forward(x, maps, traj, alpha, W))
    rhs = np.vdot(nf.nufft_adjoint(u, maps, traj, alpha, W), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_apodisation_closed_form_against_quadrature():
    """Phi(n) equals the integral of phi(u) cos(2 pi u n / G) over the window."""
    W, G = 4, 320
    beta = nf.kb_beta(W, 1.25)
    for n in (0, 17, 64, 128):
        q, _ = integrate.quad(lambda u: nf.kb_kernel(u, W, beta) * math.cos(2 * math.pi * u * n / G),
                              -W / 2, W / 2, epsabs=1e-13, epsrel=1e-13, limit=200)
        assert abs(q - nf.kb_apod(np.array([n]), G, W, beta)[0]) < 1e-10 * abs(q)


def test_grid_shape_and_beta():
    assert nf.grid_shape((256, 256), 1.25) == (320, 320)
    assert nf.grid_shape((192, 192, 192), 1.25) == (240, 240, 240)
    assert nf.grid_shape((128, 128), 2.0) == (256, 256)
    assert nf.grid_shape((255, 200), 1.25) == (320, 250)
    # Beatty's parameter is real and positive at the paper's setting
    assert 6.9 < nf.kb_beta(4, 1.25) < 7.1


def test_first_tap_is_exact_and_inside_window():
    """k0 = ceil(t - W/2) exactly, even where t - W/2 would round in float32 (tiny t)."""
    t = np.array([2.0 ** -30, 0.5, -1.0, 3.999999, -0.99999994, 0.0], dtype=np.float32)
    assert list(nf.first_tap(t, 4)) == [-1, -1, -3, 2, -2, -2]
    t = np.random.default_rng(0).uniform(-3, 3, 10000).astype(np.float32)
    t[:100] = np.float32(1e-9) * np.arange(100, dtype=np.float32)
    k0 = nf.first_tap(t, 4)
    u0 = t.astype(np.float64) - k0
    assert np.all(u0 > 1.0 - 1e-12) and np.all(u0 <= 2.0)


def test_grid_coords_are_the_rounded_exact_value():
    """t = f G / N is the float64 number nearest the exact rational value (brute force with
    fractions), so samples at +-N/2 of an odd N land exactly on the grid points +-G/2."""
    from fractions import Fraction
    rng = np.random.default_rng(5)
    img, grid = (307, 15, 64), (384, 20, 80)
    f = np.stack([rng.uniform(-n / 2, n / 2, 200) for n in img], -1).astype(np.float32)
    f[0] = [153.5, 7.5, 32.0]
    f[1] = [-153.5, -7.5, -32.0]
    t = nf.grid_coords(f, img, grid)
    for i in range(f.shape[0]):
        for d in range(3):
            assert t[i, d] == float(Fraction(float(f[i, d])) * grid[d] / img[d])
    assert list(t[0]) == [192.0, 10.0, 40.0] and list(t[1]) == [-192.0, -10.0, -40.0]
