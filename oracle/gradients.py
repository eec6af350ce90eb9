"""Oracle gradients of the NUFFT SENSE pair and of unrolled l2 PDHG (test infrastructure only).

Trajectory derivative of the Kaiser-Bessel NUFFT (Sec. 6 operator):
    d y_c[i] / d f_{i,d} = (G_d/N_d) N^{-1/2} sum_taps phi'(t_d - k_d) prod_{e != d} phi(t_e - k_e) Xhat_c[k],
    phi'(u) = I1(beta sqrt(s)) beta (-4u) / (W^2 sqrt(s)),  s = 1 - (2u/W)^2   (-> -2 beta^2 u / W^2 as s -> 0);
the tap set is held fixed (it changes only where t crosses an integer, where the kernel's
window edge makes y discontinuous in f).

For a real loss with complex gradients in the PyTorch convention g = dL/dRe + i dL/dIm:
    dL/df_{i,d} through y = A x:     Re sum_c conj(g_c[i]) dy_c[i]/df_{i,d}
    dL/df_{i,d} through x = A^H u:   Re sum_c conj(u_c[i]) d(A g_x)_c[i]/df_{i,d}
(the second follows from <g_x, d(A^H u)/df> = <FFT P^H g_x, dSpread(u)/df>).

Unrolled l2 PDHG (Sec. 4.1 with g = lambda ||x||^2/2, x_0 = xbar_0 = 0, u_0 = 0, step sizes
sigma_k, tau_k, theta_k from lambda_max and min p held constant):
    u_{k+1} = (u_k + sigma_k p (A xbar_k - y)) / (1 + sigma_k p)
    x_{k+1} = (x_k - tau_k A^H u_{k+1}) / (1 + tau_k lambda)
    xbar_{k+1} = x_{k+1} + theta_k (x_{k+1} - x_k)
and its reverse-mode sweep over the stored iterates.

Parity: pinned by tests/test_oracle_gradients.py (central finite differences of the oracle's
own forward maps; exact adjointness of the linear map y -> x_K).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy import special

from . import nufft as nf
from . import solvers as sv

__all__ = ["kb_kernel_deriv", "nufft_forward_dtraj", "traj_grad_forward", "traj_grad_adjoint",
           "unrolled_pdhg_l2", "unrolled_pdhg_l2_grad"]


def kb_kernel_deriv(u, W, beta):
    """phi'(u) on |u| <= W/2 (zero outside)."""
    u = np.asarray(u, dtype=np.float64)
    s = 1.0 - (2.0 * u / W) ** 2
    out = np.zeros_like(u)
    inside = s > 1e-12
    z = beta * np.sqrt(s[inside])
    out[inside] = special.i1(z) * beta * (-4.0 * u[inside]) / (W * W * np.sqrt(s[inside]))
    edge = (s >= 0) & ~inside
    out[edge] = -2.0 * beta * beta * u[edge] / (W * W)
    return out


def _grid_spectrum(x, maps, oversamp, W):
    img_shape = x.shape
    d = len(img_shape)
    gshape = nf.grid_shape(img_shape, oversamp)
    img = maps.astype(np.complex128) * x.astype(np.complex128)[None] / nf._apod_image(img_shape, gshape, W)[None]
    grid = np.zeros((maps.shape[0],) + gshape, dtype=np.complex128)
    grid[(slice(None),) + nf._pad_index(img_shape, gshape)] = img
    return np.fft.fftn(grid, axes=tuple(range(1, d + 1))).reshape(maps.shape[0], -1), gshape


def nufft_forward_dtraj(x, maps, traj, oversamp=1.25, W=4):
    """d y_c[i] / d f_{i,d} for the NUFFT forward: complex array [C, M, D]."""
    img_shape = x.shape
    D = len(img_shape)
    N = int(np.prod(img_shape))
    Xhat, gshape = _grid_spectrum(x, maps, oversamp, W)
    t = nf.grid_coords(traj, img_shape, gshape)
    k0 = nf.first_tap(t, W)
    M = t.shape[0]
    w, dw, idx = [], [], []
    for d in range(D):
        beta = nf.kb_beta(W, gshape[d] / img_shape[d])
        w.append([nf.kb_kernel(t[:, d] - (k0[:, d] + j), W, beta) for j in range(W)])
        dw.append([kb_kernel_deriv(t[:, d] - (k0[:, d] + j), W, beta) for j in range(W)])
        idx.append([np.mod(k0[:, d] + j, gshape[d]) for j in range(W)])
    out = np.zeros((maps.shape[0], M, D), dtype=np.complex128)
    for combo in itertools.product(range(W), repeat=D):
        flat = np.zeros(M, dtype=np.int64)
        for d, j in enumerate(combo):
            flat = flat * gshape[d] + idx[d][j]
        vals = Xhat[:, flat]
        for d in range(D):
            f = np.ones(M)
            for e, j in enumerate(combo):
                f = f * (dw[e][j] if e == d else w[e][j])
            out[:, :, d] += vals * (f * gshape[d] / img_shape[d])[None, :]
    return out / math.sqrt(N)


def traj_grad_forward(x, maps, traj, gy, oversamp=1.25, W=4):
    """dL/df through y = A x given g_y: [M, D] real."""
    Dy = nufft_forward_dtraj(x, maps, traj, oversamp, W)
    return np.real(np.sum(np.conj(gy)[:, :, None] * Dy, axis=0))


def traj_grad_adjoint(u, maps, traj, gx, oversamp=1.25, W=4):
    """dL/df through x = A^H u given g_x: [M, D] real."""
    return traj_grad_forward(gx, maps, traj, u, oversamp, W)


def unrolled_pdhg_l2(y, maps, traj, p, lam, iters, L, oversamp=1.25, W=4):
    """Forward of the unrolled l2 PDHG; returns (x_K, tape of per-iteration iterates)."""
    m = maps.astype(np.complex128)
    A = lambda v: nf.nufft_forward(v, m, traj, oversamp, W)
    AH = lambda u: nf.nufft_adjoint(u, m, traj, oversamp, W)
    y = np.asarray(y, dtype=np.complex128)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), y.shape)
    x = np.zeros(maps.shape[1:], dtype=np.complex128)
    xbar = x.copy()
    u = np.zeros_like(y)
    sched = sv.pdhg_schedule(iters, L, float(p.min()))
    tape = []
    for k in range(iters):
        sig, tau, theta = sched[k]
        u_new = (u + sig * p * (A(xbar) - y)) / (1.0 + sig * p)
        x_new = (x - tau * AH(u_new)) / (1.0 + tau * lam)
        tape.append(dict(xbar=xbar, x=x, u_new=u_new, x_new=x_new))
        xbar = x_new + theta * (x_new - x)
        x, u = x_new, u_new
    return x, dict(tape=tape, sched=sched)


def unrolled_pdhg_l2_grad(gx_K, y, maps, traj, p, lam, iters, L, tape, oversamp=1.25, W=4, want_traj=True):
    """Reverse-mode sweep: gradients of a real loss w.r.t. y (complex, [C, M]), lambda (real)
    and the trajectory ([M, D]) given g = dL/dx_K."""
    m = maps.astype(np.complex128)
    A = lambda v: nf.nufft_forward(v, m, traj, oversamp, W)
    AH = lambda u: nf.nufft_adjoint(u, m, traj, oversamp, W)
    y = np.asarray(y, dtype=np.complex128)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), y.shape)
    sched = tape["sched"]
    gx = np.array(gx_K, dtype=np.complex128)
    gxb = np.zeros_like(gx)
    gu = np.zeros_like(y)
    gy = np.zeros_like(y)
    glam = 0.0
    gf = np.zeros(np.asarray(traj).shape)
    for k in reversed(range(iters)):
        sig, tau, theta = sched[k]
        st = tape["tape"][k]
        c = 1.0 / (1.0 + tau * lam)
        alpha = 1.0 / (1.0 + sig * p)
        beta = sig * p / (1.0 + sig * p)
        gx_next = gx + (1.0 + theta) * gxb          # total gradient w.r.t. x_{k+1}
        gx_k = -theta * gxb
        glam += float(np.real(np.vdot(gx_next, -tau * c * st["x_new"])))
        gv = c * gx_next
        gx_k = gx_k + gv
        gu_next = gu - tau * A(gv)                  # total gradient w.r.t. u_{k+1}
        if want_traj:
            gf += -tau * traj_grad_adjoint(st["u_new"], maps, traj, gv, oversamp, W)
        gu = alpha * gu_next
        gr = beta * gu_next
        gxb = AH(gr)
        gy = gy - gr
        if want_traj:
            gf += traj_grad_forward(st["xbar"], maps, traj, gr, oversamp, W)
        gx = gx_k
    return gy, glam, gf
