"""Pins of the oracle's l2 solve through the dual (appendix on the connection to Trzasko et al.):
(A A^H + lambda I) w = lambda y by conjugate gradients preconditioned by the diagonal P, and
x = A^H w / lambda.  Checked against dense solves of the dual system and of the primal ridge
problem (the push-through identity A^H (A A^H + lambda I)^{-1} = (A^H A + lambda I)^{-1} A^H),
against the oracle's CG on the primal normal equations for a NUFFT problem, and against the
dual variable of the Sec. 4.1 PDHG at its fixed point (u = A x - y = -w)."""
import numpy as np
import pytest

from oracle import solvers as osv, nufft as onf
import synth


def _dense(seed=0, M=50, N=30):
    rng = np.random.default_rng(seed)
    Am = (rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))) / np.sqrt(M)
    y = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    p = rng.uniform(0.3, 2.0, M)
    return Am, (lambda x: Am @ x), (lambda u: Am.conj().T @ u), y, p


@pytest.mark.parametrize("precond", [False, True])
def test_dual_pcg_dense_solves(precond):
    Am, A, AH, y, p, = _dense()
    lam = 0.3
    pp = p if precond else 1.0
    x, w, res = osv.dual_l2_pcg(A, AH, y, pp, lam, 200, tol=1e-14)
    M, N = Am.shape
    w_ref = np.linalg.solve(Am @ Am.conj().T + lam * np.eye(M), lam * y)
    x_ref = np.linalg.solve(Am.conj().T @ Am + lam * np.eye(N), Am.conj().T @ y)
    assert np.linalg.norm(w - w_ref) < 1e-12 * np.linalg.norm(w_ref)
    assert np.linalg.norm(x - x_ref) < 1e-12 * np.linalg.norm(x_ref)
    assert res[-1] <= 1e-14 * res[0]


def test_dual_is_minus_pdhg_dual():
    """Sec. 4.1's PDHG keeps u -> A x - y; the appendix's dual variable is w = -u."""
    Am, A, AH, y, p = _dense(1)
    lam = 0.3
    x, w, _ = osv.dual_l2_pcg(A, AH, y, p, lam, 200, tol=1e-14)
    L = float(np.linalg.eigvalsh(Am.conj().T @ (p[:, None] * Am)).max())
    xp, u, _, _ = osv.pdhg(A, AH, y, p, (Am.shape[1],), "l2", lam, 10000, L)
    assert np.linalg.norm(u + w) < 2e-3 * np.linalg.norm(w)
    assert np.linalg.norm(xp - x) < 2e-3 * np.linalg.norm(x)


def test_dual_pcg_nufft_matches_primal_cg():
    w = synth.Workload("s", (24, 24), 2, 1.25, 4, "l2", 1e-2, 50, 0, "spiral",
                       dict(n_interleaves=4, n_samples=600, kmax=12.0), seed=3)
    x0, maps, traj = w.phantom(), w.maps().astype(np.complex128), w.traj()
    A = lambda v: onf.nufft_forward(v, maps, traj, 1.25, 4)
    AH = lambda u: onf.nufft_adjoint(u, maps, traj, 1.25, 4)
    y = A(x0.astype(np.complex128))
    lam = 1e-2
    x_cg = osv.cg_l2(A, AH, y, lam, x0.shape, iters=500, tol=1e-13)
    x_cg = x_cg[0] if isinstance(x_cg, tuple) else x_cg
    x, _, res = osv.dual_l2_pcg(A, AH, y, 1.0, lam, 400)
    assert res[-1] <= 1e-8 * res[0]
    assert np.linalg.norm(x - x_cg) < 1e-7 * np.linalg.norm(x_cg)
