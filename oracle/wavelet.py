"""Oracle orthonormal Daubechies-4 wavelet transform W (test infrastructure only).

Sec. 2 (Eq. obj) takes W unitary; Sec. 6 names the Daubechies-4 wavelet.  Reading used
here: the 8-tap extremal-phase Daubechies filter with 4 vanishing moments, periodised so
that W is exactly unitary, applied separably along every axis, multilevel on the
approximation block (Mallat layout: after each level the first half of every axis holds
the approximation, the second half the details).

Filter construction (Daubechies' spectral factorisation): with
P(y) = sum_{k<4} binom(3+k, k) y^k and y = (2 - z - 1/z)/4, each root y_r of P gives the
pair z, 1/z; keeping the root inside the unit circle,
H(z) = c (1 + z^{-1})^4 prod_r (1 - z_r z^{-1}),  normalised so that sum_n h[n] = sqrt(2).

One analysis level along an axis of even length L (indices mod L):
    a[k] = sum_{n=0}^{7} h[n] x[2k + n],    d[k] = sum_{n=0}^{7} g[n] x[2k + n],
    g[n] = (-1)^n h[7 - n];
synthesis is the exact transpose.

Parity: pinned by tests/test_oracle_wavelet.py (filter orthonormality and vanishing
moments, minimum phase, perfect reconstruction, norm preservation, Haar special case
checked by hand).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["daubechies_filter", "dwt_level_axis", "idwt_level_axis", "dwt", "idwt",
           "soft_threshold", "prox_l1_wavelet"]


def daubechies_filter(p=4):
    """Extremal-phase Daubechies scaling filter with p vanishing moments (2p taps)."""
    coeffs = [math.comb(p - 1 + k, k) for k in range(p)]     # ascending powers of y
    zs = []
    if p > 1:
        yr = np.roots(coeffs[::-1])
        for y in yr:
            b = 2.0 - 4.0 * y
            disc = np.sqrt(b * b - 4.0 + 0j)
            z1 = (b + disc) / 2.0
            z2 = (b - disc) / 2.0
            zs.append(z1 if abs(z1) < 1.0 else z2)
    poly = np.array([1.0 + 0j])
    for _ in range(p):
        poly = np.convolve(poly, [1.0, 1.0])
    for z in zs:
        poly = np.convolve(poly, [1.0, -z])
    h = np.real(poly)
    return h * (math.sqrt(2.0) / h.sum())


def _qmf(h):
    L = len(h)
    return np.array([(-1) ** n * h[L - 1 - n] for n in range(L)])


def dwt_level_axis(x, axis, h):
    """One analysis level along ``axis`` (periodised): returns concat(a, d) on that axis."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, 0)
    L = x.shape[0]
    g = _qmf(h)
    K = L // 2
    a = np.zeros((K,) + x.shape[1:], dtype=np.complex128)
    d = np.zeros_like(a)
    for k in range(K):
        for n in range(len(h)):
            a[k] += h[n] * x[(2 * k + n) % L]
            d[k] += g[n] * x[(2 * k + n) % L]
    return np.moveaxis(np.concatenate([a, d], axis=0), 0, axis)


def idwt_level_axis(c, axis, h):
    """Transpose of dwt_level_axis."""
    c = np.moveaxis(np.asarray(c, dtype=np.complex128), axis, 0)
    L = c.shape[0]
    K = L // 2
    g = _qmf(h)
    x = np.zeros_like(c)
    for k in range(K):
        for n in range(len(h)):
            x[(2 * k + n) % L] += h[n] * c[k] + g[n] * c[K + k]
    return np.moveaxis(x, 0, axis)


def dwt(x, levels, h=None):
    """Multilevel separable periodised DWT (Mallat layout)."""
    h = daubechies_filter(4) if h is None else h
    out = np.array(x, dtype=np.complex128)
    shape = out.shape
    for lev in range(levels):
        blk = tuple(slice(0, n >> lev) for n in shape)
        sub = out[blk]
        for ax in range(len(shape)):
            sub = dwt_level_axis(sub, ax, h)
        out[blk] = sub
    return out


def idwt(c, levels, h=None):
    """Inverse (= adjoint) of dwt."""
    h = daubechies_filter(4) if h is None else h
    out = np.array(c, dtype=np.complex128)
    shape = out.shape
    for lev in reversed(range(levels)):
        blk = tuple(slice(0, n >> lev) for n in shape)
        sub = out[blk]
        for ax in reversed(range(len(shape))):
            sub = idwt_level_axis(sub, ax, h)
        out[blk] = sub
    return out


def soft_threshold(c, t):
    """Complex soft threshold S_t(c) = c max(0, 1 - t/|c|), with S_t(0) = 0."""
    c = np.asarray(c, dtype=np.complex128)
    mag = np.abs(c)
    scale = np.where(mag > t, 1.0 - t / np.where(mag > 0, mag, 1.0), 0.0)
    return c * scale


def prox_l1_wavelet(z, t, levels, h=None):
    """prox of t*||W x||_1 for unitary W: W^H S_t(W z); all coefficients thresholded."""
    return idwt(soft_threshold(dwt(z, levels, h), t), levels, h)
