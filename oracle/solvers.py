"""Oracle solvers: power method, preconditioned PDHG, CG and FISTA (test infrastructure only).

Preconditioned PDHG for a simple g (Sec. 4.1), iteration k:
    u <- (I + sigma_k P)^{-1} (u + sigma_k P (A xbar - y))
    x_new <- prox_{tau_k g}(x - tau_k A^H u)
    xbar <- x_new + theta_k (x_new - x)
with sigma_0 = 1, tau_0 = 1/lambda_max(P A A^H) and the accelerated schedule
    theta_k = 1/(1 + 2 sigma_k min_i p_i),  sigma_{k+1} = theta_k sigma_k,  tau_{k+1} = tau_k/theta_k.
Readings where the paper is silent: x_0 = xbar_0 = 0, u_0 = 0; theta_k is computed from
sigma_k before the k-th update; lambda_max is estimated by the power method on A^H P A
(same non-zero spectrum as P A A^H) for 30 iterations (Sec. 6) from a given start vector
(all ones by default), as ||A^H P A v|| / ||v|| at the last step, with no safety margin.

Objective (Eq. obj): F(x) = 1/2 ||A x - y||^2 + g(x), g = lambda ||x||^2 / 2 or
lambda ||W x||_1.  CG on (A^H A + lambda I) x = A^H y gives the l2 optimum; FISTA gives
an independent l1 optimum.

Parity: pinned by tests/test_oracle_solvers.py (power method against numpy.linalg.eigvalsh,
PDHG l2 against the CG solution and the KKT relations u* = A x* - y and
-A^H u* = lambda x*, PDHG l1 fixed point and agreement with FISTA, sigma*tau invariant).

PDHG for g(x) = h(G x) (Sec. 4.2, total variation h = lambda ||.||_1, G the finite-difference
operator), iteration k:
    u <- (I + sigma P)^{-1} (u + sigma P (A xbar - y))
    v <- prox_{sigma h*}(v + sigma G xbar)
    x_new <- x - tau (A^H u + G^H v)
    xbar <- x_new + theta (x_new - x)
with the fixed steps theta = 1, sigma = 1, tau = 1/(lambda_max(P A A^H) + lambda_max(G G^H)).
Readings: G is the periodic forward difference along every axis, (G x)_k[j] = x[j + e_k] - x[j],
so lambda_max(G G^H) = 4 d for even sizes (bound for odd ones); h is the anisotropic complex
l1 norm lambda sum_k sum_j |(G x)_k[j]|; the paper's prox_{tau h} in the v step is read as
prox_{sigma h*}, the projection onto {|v_i| <= lambda} (v is the dual variable of h); v_0 = 0.
Pinned by tests/test_oracle_tv.py (G^H against the adjoint identity, the spectrum of G^H G
against its closed form, the projection against the Moreau identity with the complex soft
threshold, the KKT conditions of the TV problem at convergence, lambda = 0 against least squares).

l2 through the dual (appendix on the connection to Trzasko et al.): for g = lambda ||x||^2 / 2
the dual optimum w solves (A A^H + lambda I) w = lambda y and x = A^H w / lambda.  Reading: the
paper preconditions this system by the diagonal P without naming a solver; here it is conjugate
gradients with P as the preconditioner (M^{-1} = P: the Hermitian positive definite system is
solved, P shapes the iterates), from w = 0.  In the sign convention of Sec. 4.1 (u = A x - y at
the fixed point) w = -u.  Pinned by tests/test_oracle_dual_l2.py (dense solve of the dual system,
the primal ridge solution through the push-through identity, PDHG's dual fixed point u = -w).
"""
from __future__ import annotations

import math

import numpy as np

from . import wavelet as wv

__all__ = ["power_method", "pdhg_schedule", "objective", "pdhg", "cg_l2", "pcg_l2_circulant", "fista",
           "fista_l1",
           "prox_l2", "make_prox", "grad_fd", "grad_fd_adjoint", "proj_linf_ball", "tv_norm",
           "objective_tv", "pdhg_tv", "dual_l2_pcg"]


def power_method(A, AH, p, x_shape, iters=30, v0=None):
    """lambda_max(A^H P A) by the power method; returns (L, v)."""
    v = np.ones(x_shape, dtype=np.complex128) if v0 is None else np.array(v0, dtype=np.complex128)
    v = v / np.linalg.norm(v)
    L = 0.0
    for _ in range(iters):
        w = AH(p * A(v))
        L = float(np.linalg.norm(w))      # ||A^H P A v|| with ||v|| = 1
        v = w / L
    return L, v


def pdhg_schedule(iters, L, pmin):
    """(sigma_k, tau_k, theta_k) for k = 0..iters-1 (Sec. 4.1 accelerated schedule)."""
    sig, tau = 1.0, 1.0 / L
    out = []
    for _ in range(iters):
        theta = 1.0 / (1.0 + 2.0 * sig * pmin)
        out.append((sig, tau, theta))
        sig, tau = theta * sig, tau / theta
    return out


def prox_l2(z, t, lam):
    """prox of t*lam*||x||^2/2: z / (1 + t lam)."""
    return z / (1.0 + t * lam)


def make_prox(reg, lam, levels=0):
    if reg == "l2":
        return lambda z, t: prox_l2(z, t, lam)
    if reg == "l1_wavelet":
        return lambda z, t: wv.prox_l1_wavelet(z, t * lam, levels)
    raise ValueError(reg)


def objective(A, x, y, reg, lam, levels=0):
    """F(x) = 1/2 ||A x - y||^2 + g(x)."""
    r = A(x) - y
    f = 0.5 * float(np.vdot(r, r).real)
    if reg == "l2":
        f += 0.5 * lam * float(np.vdot(x, x).real)
    else:
        f += lam * float(np.sum(np.abs(wv.dwt(x, levels))))
    return f


def pdhg(A, AH, y, p, x_shape, reg, lam, iters, L, levels=0, trace=False, state=None):
    """Preconditioned PDHG (Sec. 4.1).  Returns (x, u, xbar, objective trace or None)."""
    prox = make_prox(reg, lam, levels)
    y = np.asarray(y, dtype=np.complex128)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), y.shape)
    if state is None:
        x = np.zeros(x_shape, dtype=np.complex128)
        xbar = x.copy()
        u = np.zeros_like(y)
        k0 = 0
    else:
        x, xbar, u, k0 = (np.array(state[0], dtype=np.complex128), np.array(state[1], dtype=np.complex128),
                          np.array(state[2], dtype=np.complex128), int(state[3]))
    sched = pdhg_schedule(k0 + iters, L, float(p.min()))
    objs = [] if trace else None
    for k in range(k0, k0 + iters):
        sig, tau, theta = sched[k]
        u = (u + sig * p * (A(xbar) - y)) / (1.0 + sig * p)
        x_new = prox(x - tau * AH(u), tau)
        xbar = x_new + theta * (x_new - x)
        x = x_new
        if trace:
            objs.append(objective(A, x, y, reg, lam, levels))
    return x, u, xbar, objs


def cg_l2(A, AH, y, lam, x_shape, iters=500, tol=1e-13):
    """Conjugate gradient on (A^H A + lam I) x = A^H y (the l2 optimum)."""
    b = AH(y)
    x = np.zeros(x_shape, dtype=np.complex128)
    r = b.copy()
    d = r.copy()
    rr = float(np.vdot(r, r).real)
    bn = math.sqrt(float(np.vdot(b, b).real))
    for _ in range(iters):
        q = AH(A(d)) + lam * d
        a = rr / float(np.vdot(d, q).real)
        x = x + a * d
        r = r - a * q
        rr_new = float(np.vdot(r, r).real)
        if math.sqrt(rr_new) < tol * bn:
            break
        d = r + (rr_new / rr) * d
        rr = rr_new
    return x


def pcg_l2_circulant(A, AH, y, lam, x_shape, eigs, iters, trace=False):
    """Conjugate gradients on (A^H A + lam I) x = A^H y preconditioned by M = P + lam I, P the
    App. B circulant with eigenvalues `eigs` (M^{-1} v = IDFT((DFT v) / (eigs + lam))), from x = 0.
    eigs=None runs plain CG.  Returns (x, objective trace F(x_k) after each iteration or None)."""
    b = AH(np.asarray(y, dtype=np.complex128))
    minv = (lambda v: v) if eigs is None else (lambda v: np.fft.ifftn(np.fft.fftn(v) / (np.real(eigs) + lam)))
    x = np.zeros(x_shape, dtype=np.complex128)
    r = b.copy()
    z = minv(r)
    d = z.copy()
    rz = float(np.vdot(r, z).real)
    objs = [] if trace else None
    for _ in range(iters):
        q = AH(A(d)) + lam * d
        a = rz / float(np.vdot(d, q).real)
        x = x + a * d
        r = r - a * q
        z = minv(r)
        rz_new = float(np.vdot(r, z).real)
        d = z + (rz_new / rz) * d
        rz = rz_new
        if trace:
            objs.append(objective(A, x, y, "l2", lam))
    return x, objs


def fista(A, AH, y, reg, lam, x_shape, L, iters, levels=0, trace=False):
    """FISTA (Beck & Teboulle) on 1/2 ||A x - y||^2 + g(x) with step 1/L, L >= lambda_max(A^H A):
    x_{k+1} = prox_{g/L}(z_k - A^H (A z_k - y) / L), t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,
    z_{k+1} = x_{k+1} + (t_k - 1)/t_{k+1} (x_{k+1} - x_k), x_0 = z_0 = 0, t_0 = 1.
    Returns (x, objective trace or None)."""
    prox = make_prox(reg, lam, levels)
    y = np.asarray(y, dtype=np.complex128)
    x = np.zeros(x_shape, dtype=np.complex128)
    z = x.copy()
    t = 1.0
    objs = [] if trace else None
    for _ in range(iters):
        x_new = prox(z - AH(A(z) - y) / L, 1.0 / L)
        t_new = (1 + math.sqrt(1 + 4 * t * t)) / 2
        z = x_new + ((t - 1) / t_new) * (x_new - x)
        x, t = x_new, t_new
        if trace:
            objs.append(objective(A, x, y, reg, lam, levels))
    return x, objs


def fista_l1(A, AH, y, lam, x_shape, levels, iters=2000, L=None):
    """FISTA (Beck & Teboulle) for 1/2||Ax-y||^2 + lam ||W x||_1, step 1/L, L = lambda_max(A^H A)."""
    if L is None:
        L, _ = power_method(A, AH, 1.0, x_shape, iters=100)
        L *= 1.0001
    x = np.zeros(x_shape, dtype=np.complex128)
    z = x.copy()
    t = 1.0
    for _ in range(iters):
        x_new = wv.prox_l1_wavelet(z - AH(A(z) - y) / L, lam / L, levels)
        t_new = (1 + math.sqrt(1 + 4 * t * t)) / 2
        z = x_new + ((t - 1) / t_new) * (x_new - x)
        x, t = x_new, t_new
    return x


def grad_fd(x):
    """G x: periodic forward differences, (G x)_k[j] = x[j + e_k] - x[j]; shape (d,) + x.shape."""
    x = np.asarray(x)
    return np.stack([np.roll(x, -1, axis=k) - x for k in range(x.ndim)])


def grad_fd_adjoint(v):
    """G^H v = sum_k (v_k[j - e_k] - v_k[j])."""
    v = np.asarray(v)
    return sum(np.roll(v[k], 1, axis=k) - v[k] for k in range(v.shape[0]))


def proj_linf_ball(z, lam):
    """prox of sigma h* for h = lam ||.||_1 on complex entries: the projection onto |z_i| <= lam."""
    z = np.asarray(z, dtype=np.complex128)
    mag = np.abs(z)
    out = z.copy()
    big = mag > lam
    out[big] = z[big] * (lam / mag[big])
    return out


def tv_norm(x):
    """sum_k sum_j |(G x)_k[j]| (anisotropic, complex magnitude)."""
    return float(np.sum(np.abs(grad_fd(x))))


def objective_tv(A, x, y, lam):
    """F(x) = 1/2 ||A x - y||^2 + lambda ||G x||_1."""
    r = A(x) - y
    return 0.5 * float(np.vdot(r, r).real) + lam * tv_norm(x)


def pdhg_tv(A, AH, y, p, x_shape, lam, iters, L, trace=False):
    """PDHG with the TV regulariser (Sec. 4.2).  Returns (x, u, v, xbar, objective trace or None)."""
    y = np.asarray(y, dtype=np.complex128)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), y.shape)
    d = len(x_shape)
    sig, theta = 1.0, 1.0
    tau = 1.0 / (L + 4.0 * d)
    x = np.zeros(x_shape, dtype=np.complex128)
    xbar = x.copy()
    u = np.zeros_like(y)
    v = np.zeros((d,) + tuple(x_shape), dtype=np.complex128)
    objs = [] if trace else None
    for _ in range(iters):
        u = (u + sig * p * (A(xbar) - y)) / (1.0 + sig * p)
        v = proj_linf_ball(v + sig * grad_fd(xbar), lam)
        x_new = x - tau * (AH(u) + grad_fd_adjoint(v))
        xbar = x_new + theta * (x_new - x)
        x = x_new
        if trace:
            objs.append(objective_tv(A, x, y, lam))
    return x, u, v, xbar, objs


def dual_l2_pcg(A, AH, y, p, lam, iters, tol=0.0):
    """(A A^H + lam I) w = lam y by conjugate gradients preconditioned by the diagonal p, from
    w = 0; x = A^H w / lam.  Stops after `iters` iterations or when ||r|| <= tol ||lam y||.
    Returns (x, w, residual norms ||lam y - (A A^H + lam I) w|| per iteration, first at w = 0)."""
    y = np.asarray(y, dtype=np.complex128)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), y.shape)
    w = np.zeros_like(y)
    r = lam * y
    z = p * r
    d = z.copy()
    rz = float(np.vdot(r, z).real)
    res = [float(np.linalg.norm(r))]
    for _ in range(iters):
        if rz == 0.0:
            break
        q = A(AH(d)) + lam * d
        alpha = rz / float(np.vdot(d, q).real)
        w = w + alpha * d
        r = r - alpha * q
        res.append(float(np.linalg.norm(r)))
        if tol > 0 and res[-1] <= tol * res[0]:
            break
        z = p * r
        rz_new = float(np.vdot(r, z).real)
        d = z + (rz_new / rz) * d
        rz = rz_new
    return AH(w) / lam, w, res
