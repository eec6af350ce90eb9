"""Oracle forward model and its Kaiser-Bessel NUFFT approximation (test infrastructure only).

Model (Sec. 2, Eq. model_i, extended to d dimensions with a centred index):

    y_c[i] = N^{-1/2} sum_n s_c[n] x[n] exp(-i 2 pi sum_d f_{i,d} n_d / N_d),
    n_d in [-N_d/2, N_d/2),  N = prod_d N_d,  A stacks the C coils (Eq. model).

NUFFT (Sec. 6: "following Beatty et al.", oversampling 1.25, kernel width 4):
grid size G_d = ceil(alpha N_d) rounded up to even, grid coordinate
t_{i,d} = f_{i,d} * (G_d/N_d) (float64), Kaiser-Bessel kernel

    phi_d(u) = I0(beta_d sqrt(1 - (2u/W)^2)) for |u| <= W/2, else 0,
    beta_d = pi sqrt((W/a_d)^2 (a_d - 1/2)^2 - 0.8),  a_d = G_d/N_d   (Beatty 2005),

apodisation by its continuous Fourier transform

    Phi_d(n) = W sinh(sqrt(beta^2 - (pi W n/G)^2)) / sqrt(beta^2 - (pi W n/G)^2)

(sin form when the radicand is negative), zero padding with pixel n_d stored at
grid index n_d mod G_d, a forward DFT of size G, and W^d-tap interpolation with
taps k_d = ceil(t_d - W/2) + j, j = 0..W-1, evaluated as ceil(t_d) - W/2 + j (the same
integer for even W, with no rounding of t_d - W/2), read at index k_d mod G_d.  Every tap then has |t_d - k_d| <= W/2.
The adjoint is the exact transpose, step by step in reverse order.

Parity: pinned by tests/test_oracle_nufft.py (brute-force NUDFT on tiny inputs,
accuracy improving with W to < 1e-9 at W = 12, alpha = 2; adjoint identity;
Phi closed form against quadrature; on-grid NUDFT against numpy.fft).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

__all__ = [
    "grid_shape", "kb_beta", "kb_kernel", "kb_apod", "grid_coords", "first_tap",
    "nudft_matrix", "sense_matrix", "nudft_forward", "nudft_adjoint",
    "nufft_forward", "nufft_adjoint", "simulate_kspace",
]


def grid_shape(img_shape, oversamp):
    """G_d = ceil(oversamp * N_d), rounded up to an even number."""
    out = []
    for n in img_shape:
        g = int(math.ceil(oversamp * n - 1e-9))
        g += g % 2
        out.append(g)
    return tuple(out)


def kb_beta(W, a):
    """Beatty et al.'s Kaiser-Bessel shape parameter for width W and oversampling a."""
    return math.pi * math.sqrt((W / a) ** 2 * (a - 0.5) ** 2 - 0.8)


def kb_kernel(u, W, beta):
    """phi(u) = I0(beta sqrt(1-(2u/W)^2)) on |u| <= W/2, zero outside (float64)."""
    u = np.asarray(u, dtype=np.float64)
    arg = 1.0 - (2.0 * u / W) ** 2
    out = np.where(arg >= 0.0, np.i0(beta * np.sqrt(np.maximum(arg, 0.0))), 0.0)
    return out


def kb_apod(n, G, W, beta):
    """Continuous Fourier transform of phi at frequency n/G (real, even)."""
    nu = np.asarray(n, dtype=np.float64) / G
    z2 = beta * beta - (math.pi * W * nu) ** 2
    out = np.empty_like(z2)
    pos = z2 > 0
    zp = np.sqrt(z2[pos])
    out[pos] = W * np.sinh(zp) / zp
    neg = z2 < 0
    zn = np.sqrt(-z2[neg])
    out[neg] = W * np.sin(zn) / zn
    out[z2 == 0] = W
    return out


def grid_coords(traj, img_shape, gshape):
    """t_{i,d} = f_{i,d} G_d / N_d in float64 (the operator as the paper defines it), rounded
    once: f G is exact for a float32 f and an integer G below 2^29, so the division returns
    the float64 number nearest the exact t, and a t that is exactly an integer (a sample on a
    grid point, where the truncated window's first-tap choice decides which edge tap is
    taken) comes out as that integer."""
    traj = np.asarray(traj, dtype=np.float64)
    g = np.array(gshape, dtype=np.float64)[None, :]
    n = np.array(img_shape, dtype=np.float64)[None, :]
    return traj * g / n


def first_tap(t, W):
    """k0 = ceil(t) - W/2 for even W: the same integer as ceil(t - W/2) in exact arithmetic,
    computed without rounding (t - W/2 in floating point can round onto an integer when |t| is
    tiny, which would push the first tap just outside the window)."""
    t = np.asarray(t)
    return np.ceil(t).astype(np.int64) - W // 2


def _centred(n):
    return np.arange(n) - n // 2


def nudft_matrix(img_shape, traj):
    """Dense exact model matrix E[i, n] = N^{-1/2} exp(-i 2 pi sum_d f_{i,d} n_d / N_d)."""
    traj = np.asarray(traj, dtype=np.float64)
    grids = np.meshgrid(*[_centred(n) for n in img_shape], indexing="ij")
    N = int(np.prod(img_shape))
    phase = np.zeros((traj.shape[0], N))
    for d, n in enumerate(img_shape):
        phase += np.outer(traj[:, d], grids[d].ravel()) / n
    return np.exp(-2j * np.pi * phase) / math.sqrt(N)


def sense_matrix(maps, traj):
    """Dense A in C^{MC x N}: rows (c, i) = s_c[n] E[i, n], stacked coil-major (Eq. model)."""
    C = maps.shape[0]
    E = nudft_matrix(maps.shape[1:], traj)
    return np.concatenate([E * maps[c].reshape(1, -1) for c in range(C)], axis=0)


def nudft_forward(x, maps, traj):
    """Exact Eq. model_i, evaluated sample by sample (no matrix held): returns [C, M]."""
    img_shape = x.shape
    traj = np.asarray(traj, dtype=np.float64)
    N = int(np.prod(img_shape))
    grids = np.meshgrid(*[_centred(n) for n in img_shape], indexing="ij")
    sx = (maps * x[None]).reshape(maps.shape[0], -1).astype(np.complex128)
    out = np.empty((maps.shape[0], traj.shape[0]), dtype=np.complex128)
    for i in range(traj.shape[0]):
        ph = sum(traj[i, d] * grids[d].ravel() / img_shape[d] for d in range(len(img_shape)))
        out[:, i] = sx @ np.exp(-2j * np.pi * ph)
    return out / math.sqrt(N)


def nudft_adjoint(y, maps, traj):
    """Exact transpose of nudft_forward: x[n] = N^{-1/2} sum_c conj(s_c[n]) sum_i y_c[i] e^{+...}."""
    img_shape = maps.shape[1:]
    traj = np.asarray(traj, dtype=np.float64)
    N = int(np.prod(img_shape))
    grids = np.meshgrid(*[_centred(n) for n in img_shape], indexing="ij")
    acc = np.zeros((maps.shape[0], N), dtype=np.complex128)
    for i in range(traj.shape[0]):
        ph = sum(traj[i, d] * grids[d].ravel() / img_shape[d] for d in range(len(img_shape)))
        acc += y[:, i:i + 1] * np.exp(2j * np.pi * ph)[None, :]
    x = np.sum(np.conj(maps.reshape(maps.shape[0], -1)) * acc, axis=0)
    return (x / math.sqrt(N)).reshape(img_shape)


class _Taps:
    """Per-sample interpolation taps: flat grid indices [T, M] and weights [T, M]."""

    def __init__(self, traj, img_shape, gshape, W):
        d = len(img_shape)
        t = grid_coords(traj, img_shape, gshape)
        k0 = first_tap(t, W)
        per_dim_idx, per_dim_w = [], []
        for dd in range(d):
            beta = kb_beta(W, gshape[dd] / img_shape[dd])
            idx, w = [], []
            for j in range(W):
                k = k0[:, dd] + j
                w.append(kb_kernel(t[:, dd] - k, W, beta))
                idx.append(np.mod(k, gshape[dd]))
            per_dim_idx.append(idx)
            per_dim_w.append(w)
        flat, wts = [], []
        for combo in itertools.product(range(W), repeat=d):
            f = np.zeros(t.shape[0], dtype=np.int64)
            wt = np.ones(t.shape[0])
            for dd, j in enumerate(combo):
                f = f * gshape[dd] + per_dim_idx[dd][j]
                wt = wt * per_dim_w[dd][j]
            flat.append(f)
            wts.append(wt)
        self.flat = np.stack(flat)
        self.w = np.stack(wts)


def _apod_image(img_shape, gshape, W):
    """prod_d Phi_d(n_d) on the centred image grid."""
    parts = []
    for n, g in zip(img_shape, gshape):
        parts.append(kb_apod(_centred(n), g, W, kb_beta(W, g / n)))
    out = parts[0]
    for p in parts[1:]:
        out = np.multiply.outer(out, p)
    return out


def _pad_index(img_shape, gshape):
    return np.ix_(*[np.mod(_centred(n), g) for n, g in zip(img_shape, gshape)])


def nufft_forward(x, maps, traj, oversamp=1.25, W=4):
    """NUFFT approximation of A x: coil multiply, apodise, pad, DFT, interpolate. [C, M]."""
    img_shape = x.shape
    d = len(img_shape)
    gshape = grid_shape(img_shape, oversamp)
    N = int(np.prod(img_shape))
    C = maps.shape[0]
    img = maps.astype(np.complex128) * x.astype(np.complex128)[None] / _apod_image(img_shape, gshape, W)[None]
    grid = np.zeros((C,) + gshape, dtype=np.complex128)
    grid[(slice(None),) + _pad_index(img_shape, gshape)] = img
    Xhat = np.fft.fftn(grid, axes=tuple(range(1, d + 1))).reshape(C, -1)
    taps = _Taps(traj, img_shape, gshape, W)
    y = np.zeros((C, taps.w.shape[1]), dtype=np.complex128)
    for j in range(taps.w.shape[0]):
        y += taps.w[j][None, :] * Xhat[:, taps.flat[j]]
    return y / math.sqrt(N)


def nufft_adjoint(y, maps, traj, oversamp=1.25, W=4):
    """Exact transpose of nufft_forward: spread, inverse DFT (unnormalised), crop, apodise, coil combine."""
    img_shape = maps.shape[1:]
    d = len(img_shape)
    gshape = grid_shape(img_shape, oversamp)
    N = int(np.prod(img_shape))
    G = int(np.prod(gshape))
    C = maps.shape[0]
    taps = _Taps(traj, img_shape, gshape, W)
    flat = taps.flat.ravel()
    grid = np.empty((C, G), dtype=np.complex128)
    for c in range(C):
        v = (taps.w * np.asarray(y[c], dtype=np.complex128)[None, :]).ravel()
        grid[c] = np.bincount(flat, weights=v.real, minlength=G) + 1j * np.bincount(flat, weights=v.imag, minlength=G)
    grid = grid.reshape((C,) + gshape)
    img = np.fft.ifftn(grid, axes=tuple(range(1, d + 1))) * G
    img = img[(slice(None),) + _pad_index(img_shape, gshape)] / _apod_image(img_shape, gshape, W)[None]
    x = np.sum(np.conj(maps.astype(np.complex128)) * img, axis=0)
    return x / math.sqrt(N)


def simulate_kspace(x, maps, traj, noise, rel_sigma=0.01, oversamp=2.0, W=8):
    """Synthetic measurements y = A x + w: A taken as a high-accuracy NUFFT (alpha 2, W 8,
    so that the data are not made with the reconstruction's own operator), w = sigma * noise
    with sigma = rel_sigma * max|A x|."""
    y0 = nufft_forward(x, maps, traj, oversamp=oversamp, W=W)
    sigma = rel_sigma * np.max(np.abs(y0))
    return y0 + sigma * noise
