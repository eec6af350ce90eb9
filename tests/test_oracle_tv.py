"""Pins of the oracle's TV-regularised PDHG (Sec. 4.2) against facts it does not compute itself:
the adjoint identity of the finite-difference operator, the closed-form spectrum of G^H G
(periodic differences are diagonalised by the DFT), the Moreau identity linking the dual
projection to the complex soft threshold, the optimality (KKT) conditions of
min 1/2 ||Ax - y||^2 + lambda ||G x||_1 at convergence, and least squares at lambda = 0."""
import itertools

import numpy as np
import pytest

from oracle import solvers as osv


def _cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("shape", [(5, 6), (4, 3, 5), (8,)])
def test_grad_adjoint_identity(shape):
    rng = np.random.default_rng(1)
    x = _cplx(rng, shape)
    v = _cplx(rng, (len(shape),) + shape)
    lhs = np.vdot(osv.grad_fd(x), v)
    rhs = np.vdot(x, osv.grad_fd_adjoint(v))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def _dense(op, shape):
    n = int(np.prod(shape))
    cols = []
    for i in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[i] = 1.0
        cols.append(np.ravel(op(e.reshape(shape))))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("shape", [(4, 6), (3, 5), (2, 4, 6)])
def test_grad_spectrum_closed_form(shape):
    """G^H G = sum_k (2 - 2 cos(2 pi m_k / n_k)) in the DFT basis; its largest value is 4 d for
    even sizes (the step-size bound of Sec. 4.2) and smaller otherwise."""
    G = _dense(osv.grad_fd, shape)
    ev = np.sort(np.linalg.eigvalsh(G.conj().T @ G))
    closed = np.sort([sum(2.0 - 2.0 * np.cos(2.0 * np.pi * m[k] / shape[k]) for k in range(len(shape)))
                      for m in itertools.product(*[range(n) for n in shape])])
    assert np.allclose(ev, closed, atol=1e-10)
    if all(n % 2 == 0 for n in shape):
        assert abs(ev[-1] - 4.0 * len(shape)) < 1e-10
    else:
        assert ev[-1] < 4.0 * len(shape)


@pytest.mark.parametrize("sigma", [0.3, 1.0, 2.5])
def test_dual_projection_moreau(sigma):
    """prox_{sigma h*}(z) = z - sigma prox_{h/sigma}(z/sigma) with h = lambda ||.||_1, whose prox
    is the complex soft threshold S_t(c) = c max(0, 1 - t/|c|)."""
    rng = np.random.default_rng(2)
    lam = 0.7
    z = 1.5 * _cplx(rng, 200)
    t = lam / sigma
    zs = z / sigma
    soft = zs * np.maximum(0.0, 1.0 - t / np.abs(zs))
    assert np.allclose(osv.proj_linf_ball(z, lam), z - sigma * soft, atol=1e-12)


def _small_problem(seed=0):
    rng = np.random.default_rng(seed)
    shape = (6, 6)
    M, N = 60, 36
    Am = _cplx(rng, (M, N)) / np.sqrt(M)
    A = lambda x: Am @ np.ravel(x)
    AH = lambda u: (Am.conj().T @ u).reshape(shape)
    xt = np.zeros(shape, dtype=np.complex128)
    xt[1:4, 2:5] = 1 + 0.5j
    y = A(xt) + 0.05 * _cplx(rng, M)
    p = rng.uniform(0.5, 1.5, M)
    L = float(np.linalg.eigvalsh(Am.conj().T @ (p[:, None] * Am)).max())
    return Am, A, AH, y, p, L, shape


def test_pdhg_tv_kkt_at_convergence():
    """At the fixed point: u = A x - y, A^H u + G^H v = 0, |v| <= lambda, and
    v = lambda G x / |G x| wherever G x is non-zero (v in lambda times the subdifferential)."""
    Am, A, AH, y, p, L, shape = _small_problem()
    lam = 0.2
    x, u, v, _, objs = osv.pdhg_tv(A, AH, y, p, shape, lam, 3000, L, trace=True)
    r = A(x) - y
    assert np.linalg.norm(u - r) < 1e-9 * np.linalg.norm(r)
    assert np.linalg.norm(AH(u) + osv.grad_fd_adjoint(v)) < 1e-9 * np.linalg.norm(AH(u))
    assert np.abs(v).max() <= lam * (1 + 1e-12)
    g = osv.grad_fd(x)
    mag = np.abs(g)
    big = mag > 1e-6
    assert big.sum() > 0
    assert np.abs(v[big] - lam * g[big] / mag[big]).max() < 1e-8 * lam
    # the objective settles at the optimum it reports
    assert abs(objs[-1] - osv.objective_tv(A, x, y, lam)) < 1e-12 * objs[-1]
    assert objs[-1] <= min(objs) * (1 + 1e-12)


def test_pdhg_tv_lambda_zero_is_least_squares():
    Am, A, AH, y, p, L, shape = _small_problem(3)
    x, _, v, _, _ = osv.pdhg_tv(A, AH, y, p, shape, 0.0, 4000, L)
    x_ls = np.linalg.lstsq(Am, y, rcond=None)[0].reshape(shape)
    assert np.abs(v).max() == 0.0
    assert np.linalg.norm(x - x_ls) < 1e-8 * np.linalg.norm(x_ls)


def test_pdhg_tv_step_sizes():
    """tau (lambda_max(P A A^H) + lambda_max(G G^H)) = 1 with sigma = theta = 1: one iteration
    from zero gives x_1 = -tau (A^H u_1 + G^H v_1) with u_1 = -p y / (1 + p), v_1 = 0."""
    Am, A, AH, y, p, L, shape = _small_problem(4)
    x1, u1, v1, xb1, _ = osv.pdhg_tv(A, AH, y, p, shape, 0.1, 1, L)
    tau = 1.0 / (L + 8.0)
    assert np.allclose(u1, -p * y / (1 + p), atol=1e-14)
    assert np.abs(v1).max() == 0.0
    assert np.allclose(x1, -tau * AH(u1), atol=1e-14)
    assert np.allclose(xb1, 2 * x1, atol=1e-14)
