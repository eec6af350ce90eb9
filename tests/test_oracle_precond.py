"""Pins of the oracle's diagonal k-space preconditioners (no GPU).

Sec. 5 (general form, Eq. sc_precond, Eq. mc_precond), Sec. 5.1 (fast route, Fig. 2)
and App. A (argmin derivation).
"""
import os

import numpy as np
import pytest

from oracle import nufft as nf
from oracle import precond as pc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _problem(shape=(8, 6), C=2, M=30, seed=2):
    rng = np.random.default_rng(seed)
    maps = rng.standard_normal((C,) + shape) + 1j * rng.standard_normal((C,) + shape)
    traj = np.stack([rng.uniform(-n / 2, n / 2, M) for n in shape], -1).astype(np.float32)
    return maps, traj


def test_cartesian_single_channel_is_one():
    """Golden (Sec. 5): p = 1 on a full Cartesian grid."""
    data = np.loadtxt(os.path.join(GOLDEN, "cartesian_sc.txt"))
    traj = data[:, :2].astype(np.float32)
    expected = data[:, 2]
    A = nf.sense_matrix(np.ones((1, 8, 6)), traj)
    assert np.abs(pc.precond_bruteforce(A) - expected).max() < 1e-12
    assert np.abs(pc.sc_precond_dirichlet(traj, (8, 6)) - expected).max() < 1e-12
    assert np.abs(pc.sc_precond_fast(traj, (8, 6), exact=True) - expected).max() < 1e-12


def test_single_channel_dirichlet_closed_form():
    """The sum over n of Eq. sc_precond equals the sinc^2 / Dirichlet closed form (with 1/N^2)."""
    _, traj = _problem()
    A = nf.sense_matrix(np.ones((1, 8, 6)), traj)
    assert np.abs(pc.sc_precond_dirichlet(traj, (8, 6)) - pc.precond_bruteforce(A)).max() < 1e-12


def test_mc_formula_matches_bruteforce():
    maps, traj = _problem()
    pb = pc.precond_bruteforce(nf.sense_matrix(maps, traj)).reshape(2, -1)
    assert np.abs(pc.mc_precond_direct(maps, traj) - pb).max() < 1e-12 * pb.max()


def test_fast_route_exact_matches_bruteforce():
    """Autocorrelation/PSF route (Sec. 5.1) with exact sums reproduces the general form."""
    maps, traj = _problem(shape=(6, 7), C=3, M=25, seed=4)
    pb = pc.precond_bruteforce(nf.sense_matrix(maps, traj)).reshape(3, -1)
    assert np.abs(pc.mc_precond_fast(maps, traj, exact=True) - pb).max() < 1e-11 * pb.max()


def test_fast_route_nufft_converges():
    maps, traj = _problem()
    pb = pc.precond_bruteforce(nf.sense_matrix(maps, traj)).reshape(2, -1)
    e12 = np.abs(pc.mc_precond_fast(maps, traj, 2.0, 12) - pb).max() / pb.max()
    e4 = np.abs(pc.mc_precond_fast(maps, traj, 1.25, 4) - pb).max() / pb.max()
    assert e12 < 1e-9
    assert e4 < 2e-2


def test_fast_route_3d():
    maps, traj = _problem(shape=(4, 6, 4), C=2, M=20, seed=5)
    pb = pc.precond_bruteforce(nf.sense_matrix(maps, traj)).reshape(2, -1)
    assert np.abs(pc.mc_precond_fast(maps, traj, exact=True) - pb).max() < 1e-11 * pb.max()


def test_sc_equals_mc_with_unit_single_coil():
    """Fig. 2 caption: SC is MC with C = 1 and s_1 all ones."""
    _, traj = _problem()
    a = pc.sc_precond_fast(traj, (8, 6), exact=True)
    b = pc.mc_precond_direct(np.ones((1, 8, 6)), traj)[0]
    assert np.abs(a - b).max() < 1e-12


def test_autocorrelation_of_ones_is_triangle():
    r = pc.autocorrelation_sum(np.ones((1, 6, 4)))[0]
    ky, kx = np.meshgrid(np.arange(-6, 6), np.arange(-4, 4), indexing="ij")
    tri = np.maximum(6 - np.abs(ky), 0) * np.maximum(4 - np.abs(kx), 0)
    assert np.abs(r - tri).max() < 1e-11


def test_argmin_property():
    """App. A: the returned p minimises ||diag(p) A A^H - I||_F; perturbations raise it."""
    maps, traj = _problem(M=12)
    A = nf.sense_matrix(maps, traj)
    p = pc.precond_bruteforce(A)
    J0 = pc.precond_objective(p, A)
    rng = np.random.default_rng(9)
    for _ in range(10):
        q = p.copy()
        i = rng.integers(len(p))
        q[i] *= 1 + rng.choice([-1, 1]) * 0.05
        assert pc.precond_objective(q, A) > J0


def test_printed_sc_prefactor_is_off_by_n():
    """Reading of Eq. sc_precond: the printed 1/N would make p N times smaller than the
    general form; the oracle follows the general form (1/N^2)."""
    _, traj = _problem()
    A = nf.sense_matrix(np.ones((1, 8, 6)), traj)
    pb = pc.precond_bruteforce(A)
    E = nf.nudft_matrix((8, 6), traj) * np.sqrt(48)
    S = E @ E.conj().T
    printed = 48.0 / np.sum(np.abs(S) ** 2, axis=1)   # 1 / ((1/N) sum |.|^2)
    assert np.allclose(printed * 48, pb)
