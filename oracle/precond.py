"""Oracle l2-optimised diagonal k-space preconditioners (test infrastructure only).

Sec. 5 and App. A: p = argmin_p ||diag(p) A A^H - I||_F^2, solved row by row as

    p[r]^{-1} = sum_j |a_r^H a_j|^2 / ||a_r||^2                          (general form)

* single-channel (Eq. sc_precond): a_i[n] = e^{-i 2 pi f_i n/N}/sqrt(N); the paper
  prints a 1/N prefactor, but the general form with ||a_i||^2 = 1 gives 1/N^2, which is
  also what Eq. mc_precond gives for C = 1, s = 1, and the only factor that yields
  p = 1 on a full Cartesian grid (Sec. 5).  The oracle uses 1/N^2.
* multi-channel (Eq. mc_precond): p_c[i]^{-1} = 1/(||s_c||^2 N) sum_j sum_d
  |sum_n s_c[n] s_d^*[n] e^{-i 2 pi (f_i - f_j) n / N}|^2.
* fast route (Sec. 5.1, Fig. 2): r_cd = autocorrelation of q_cd = s_c s_d^* (FFT on a
  2N grid), h[k] = N^{-1/2} sum_j e^{+i 2 pi f_j k/N} (a type-1 NUFFT of ones at 2 f_j on
  the 2N grid), p_c[i]^{-1} = 1/(||s_c||^2 sqrt(N)) sum_k sum_d r_cd[k] h[k]
  e^{-i 2 pi f_i k / N} (a type-2 NUFFT at 2 f_i); the real part is taken.

Parity: pinned by tests/test_oracle_precond.py (dense brute force, the Dirichlet closed
form, p = 1 for Cartesian sampling, SC == MC with C = 1 and s = 1, the triangle
autocorrelation of an all-ones image, the argmin property, and fast vs brute force).

l2-optimised circulant preconditioner (App. B, the comparison system of Sec. 6):
P = argmin over circulant P of ||A^H A - P||_F^2, P[m, n] = c[(m - n) mod N] (modulo per axis),
solved diagonal by diagonal: c[k] = 1/N sum over the pairs (m, n) with (m - n) mod N = k of
(A^H A)[m, n].  With r[k] = N^{-1/2} sum_c sum_{m - n = k} s_c^*[m] s_c[n] and the point-spread
function h of Sec. 5.1, every pair with m - n = d contributes r[d] h[d] / N in total, so
c[k] = 1/N sum over the lags d = k - s N (s in {0, 1} per axis) of r[d] h[d].  Reading: the
appendix prints c[k] = r[k] h[k] + r[k - N] h[k - N] without the 1/N that its own averaging over
the N entries of a circulant diagonal produces; the argmin is used here (a uniform scale, which
preconditioned CG does not see).  Pinned by tests/test_oracle_circulant.py (the dense argmin,
its normal equations, the identity for fully sampled Cartesian k-space with one unit coil,
Hermitian symmetry, and PCG reaching the CG optimum).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import nufft as nf

__all__ = [
    "precond_bruteforce", "sc_precond_dirichlet", "mc_precond_direct",
    "autocorrelation_sum", "psf_h", "mc_precond_fast", "sc_precond_fast",
    "precond_objective", "circulant_kernel_bruteforce", "coil_autocorrelation", "circulant_kernel",
    "circulant_eigenvalues", "circulant_objective",
]


def precond_bruteforce(A):
    """p[r] = ||a_r||^2 / sum_j |a_r^H a_j|^2 from a dense A (rows a_r)."""
    G = A @ A.conj().T
    return np.real(np.diag(G)) / np.sum(np.abs(G) ** 2, axis=1)


def precond_objective(p, A):
    """||diag(p) A A^H - I||_F^2 (App. A objective, without the 1/2)."""
    G = A @ A.conj().T
    return float(np.sum(np.abs(p[:, None] * G - np.eye(G.shape[0])) ** 2))


def sc_precond_dirichlet(traj, img_shape):
    """Single-channel p via the closed form prod_d |sin(pi D_d)/sin(pi D_d/N_d)|^2 / N^2,
    D = f_i - f_j; the removable singularities (D_d/N_d integer) take the limit N_d."""
    traj = np.asarray(traj, dtype=np.float64)
    N = float(np.prod(img_shape))
    tot = np.ones((traj.shape[0], traj.shape[0]))
    for d, n in enumerate(img_shape):
        D = traj[:, d][:, None] - traj[:, d][None, :]
        den = np.sin(np.pi * D / n)
        num = np.sin(np.pi * D)
        sing = np.abs(den) < 1e-12
        ratio = np.where(sing, float(n), num / np.where(sing, 1.0, den))
        tot *= ratio ** 2
    return N * N / np.sum(tot, axis=1)


def mc_precond_direct(maps, traj):
    """Eq. mc_precond summed term by term (O(M^2 N C^2)); returns p [C, M]."""
    img_shape = maps.shape[1:]
    C = maps.shape[0]
    N = int(np.prod(img_shape))
    traj = np.asarray(traj, dtype=np.float64)
    M = traj.shape[0]
    E = nf.nudft_matrix(img_shape, traj) * math.sqrt(N)      # e^{-i 2 pi f_i n / N}
    s = maps.reshape(C, -1).astype(np.complex128)
    p = np.empty((C, M))
    for c in range(C):
        acc = np.zeros(M)
        for d in range(C):
            q = s[c] * np.conj(s[d])
            # S[i, j] = sum_n q[n] e^{-i 2 pi (f_i - f_j) n / N}
            S = (E * q[None, :]) @ np.conj(E).T
            acc += np.sum(np.abs(S) ** 2, axis=1)
        p[c] = np.sum(np.abs(s[c]) ** 2) * N / acc
    return p


def _ones_maps(shape):
    return np.ones((1,) + tuple(shape), dtype=np.complex128)


def autocorrelation_sum(maps):
    """r_c[k] = sum_d r_cd[k], r_cd[k] = sum_{m-n=k} conj(q_cd[n]) q_cd[m], q_cd = s_c s_d^*,
    computed by FFT on the zero-padded 2N grid.  Returned centred: index k_d + N_d holds lag
    k_d in [-N_d, N_d).  Shape [C, 2N_1, ..., 2N_d]."""
    img_shape = maps.shape[1:]
    d = len(img_shape)
    C = maps.shape[0]
    big = tuple(2 * n for n in img_shape)
    axes = tuple(range(1, d + 1))
    idx = np.ix_(*[np.mod(np.arange(n) - n // 2, 2 * n) for n in img_shape])
    s = maps.astype(np.complex128)
    R = np.zeros((C,) + big)
    for c in range(C):
        for dd in range(C):
            q = np.zeros(big, dtype=np.complex128)
            q[idx] = s[c] * np.conj(s[dd])
            R[c] += np.abs(np.fft.fftn(q)) ** 2
    r = np.fft.ifftn(R, axes=axes)
    return np.fft.fftshift(r, axes=axes)


def psf_h(traj, img_shape, oversamp=1.25, W=4, exact=False):
    """h[k] = N^{-1/2} sum_j e^{+i 2 pi sum_d f_{j,d} k_d / N_d} on k_d in [-N_d, N_d), centred.

    exact=False: type-1 NUFFT of ones at coordinates 2 f_j on the 2N image (what the method
    does); exact=True: the sum evaluated directly (for tests)."""
    N = int(np.prod(img_shape))
    big = tuple(2 * n for n in img_shape)
    traj = np.asarray(traj, dtype=np.float64)
    M = traj.shape[0]
    if exact:
        return nf.nudft_adjoint(np.ones((1, M)), _ones_maps(big), 2.0 * traj) * math.sqrt(2 ** len(img_shape))
    traj2 = 2.0 * traj
    hb = nf.nufft_adjoint(np.ones((1, M)), _ones_maps(big), traj2, oversamp, W)
    # adjoint on the 2N image carries (2^d N)^{-1/2}; h carries N^{-1/2}
    return hb * math.sqrt(np.prod(big) / N)


def mc_precond_fast(maps, traj, oversamp=1.25, W=4, exact=False):
    """Sec. 5.1 fast route; returns p [C, M] (float64).  exact=True replaces both NUFFTs by
    direct sums, which leaves only the FFT autocorrelation (exact) in the chain."""
    img_shape = maps.shape[1:]
    C = maps.shape[0]
    N = int(np.prod(img_shape))
    big = tuple(2 * n for n in img_shape)
    traj = np.asarray(traj, dtype=np.float64)
    r = autocorrelation_sum(maps)
    h = psf_h(traj, img_shape, oversamp, W, exact=exact)
    traj2 = 2.0 * traj
    ones = _ones_maps(big)
    p = np.empty((C, traj.shape[0]))
    for c in range(C):
        v = r[c] * h
        if exact:
            s = nf.nudft_forward(v, ones, traj2)[0]
        else:
            s = nf.nufft_forward(v, ones, traj2, oversamp, W)[0]
        s = s * math.sqrt(np.prod(big))
        norm2 = float(np.sum(np.abs(maps[c].astype(np.complex128)) ** 2))
        p[c] = norm2 * math.sqrt(N) / np.real(s)
    return p


def sc_precond_fast(traj, img_shape, oversamp=1.25, W=4, exact=False):
    """Single-channel preconditioner: the fast route with C = 1 and s = 1 (Fig. 2 caption). [M]."""
    return mc_precond_fast(_ones_maps(img_shape), traj, oversamp, W, exact=exact)[0]


def _lag_index(img_shape):
    """Flat image index -> multi-index, for the brute-force diagonal sums."""
    return np.stack(np.unravel_index(np.arange(int(np.prod(img_shape))), img_shape), axis=-1)


def circulant_kernel_bruteforce(A, img_shape):
    """App. B argmin from a dense A: c[k] = 1/N sum over (m, n) with (m - n) mod N = k (per axis)
    of (A^H A)[m, n].  Returned with index k_d in [0, N_d) (array position k)."""
    H = A.conj().T @ A
    N = int(np.prod(img_shape))
    idx = _lag_index(img_shape)
    c = np.zeros(img_shape, dtype=np.complex128)
    lag = np.mod(idx[:, None, :] - idx[None, :, :], np.array(img_shape))
    np.add.at(c, tuple(lag[..., d].ravel() for d in range(len(img_shape))), H.ravel())
    return c / N


def circulant_objective(c, A, img_shape):
    """||A^H A - P||_F^2 for the circulant P[m, n] = c[(m - n) mod N]."""
    H = A.conj().T @ A
    idx = _lag_index(img_shape)
    lag = np.mod(idx[:, None, :] - idx[None, :, :], np.array(img_shape))
    P = c[tuple(lag[..., d] for d in range(len(img_shape)))]
    return float(np.sum(np.abs(H - P) ** 2))


def coil_autocorrelation(maps):
    """r[k] = N^{-1/2} sum_c sum_{m - n = k} s_c^*[m] s_c[n] for lags k_d in [-N_d, N_d), by FFT on
    the zero-padded 2N grid; returned centred (array position k_d + N_d holds lag k_d)."""
    img_shape = maps.shape[1:]
    d = len(img_shape)
    N = int(np.prod(img_shape))
    big = tuple(2 * n for n in img_shape)
    R = np.zeros(big)
    for c in range(maps.shape[0]):
        q = np.zeros(big, dtype=np.complex128)
        q[tuple(slice(0, n) for n in img_shape)] = maps[c]
        R += np.abs(np.fft.fftn(q)) ** 2
    # IFFT of |S|^2 is sum_n s[n + k] s^*[n]; the conjugate-mirrored lag gives sum_n s^*[n + k] s[n]
    rho = np.fft.ifftn(R)
    r = np.conj(rho)
    return np.fft.fftshift(r) / math.sqrt(N)


def circulant_kernel(maps, traj, oversamp=1.25, W=4, exact=False):
    """App. B through r and h: c[k] = 1/N sum over s in {0, 1}^d of r[k - s N] h[k - s N], k_d in
    [0, N_d); h as in Sec. 5.1 (exact=True: the direct sum; else the type-1 NUFFT of ones)."""
    img_shape = maps.shape[1:]
    N = int(np.prod(img_shape))
    r = coil_autocorrelation(maps.astype(np.complex128))
    h = psf_h(traj, img_shape, oversamp, W, exact=exact)
    rh = r * h                                        # centred: position k + N_d holds lag k
    c = np.zeros(img_shape, dtype=np.complex128)
    for shift in itertools.product((0, 1), repeat=len(img_shape)):
        # lag k - s N for k in [0, N): position k - s N + N = k + (1 - s) N
        sl = tuple(slice((1 - s) * n, (1 - s) * n + n) for s, n in zip(shift, img_shape))
        c += rh[sl]
    return c / N


def circulant_eigenvalues(c):
    """Eigenvalues of the (multi-level) circulant P[m, n] = c[(m - n) mod N]: the DFT of c, real
    for the Hermitian P that A^H A gives."""
    return np.fft.fftn(c)
