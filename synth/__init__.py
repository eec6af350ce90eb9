"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 6, "Dataset Details").

The paper's liver, cardiac, brain and 3D UTE datasets and its ESPIRiT coil maps
are not available, so every run uses inputs drawn here from
``numpy.random.default_rng(seed)``:

* a random-ellipse (ellipsoid in 3D) phantom with a smooth global phase,
* Gaussian-bump coil sensitivity maps normalised to unit sum-of-squares,
* golden-angle radial, variable-density Archimedean spiral and 3D
  Fibonacci-sphere centre-out radial trajectories, in cycles/FOV,
* unit-variance complex Gaussian noise (scaled by the caller),
* the descriptor list of the batched multi-case workload.

This module holds no arithmetic of the reconstruction method itself (no
Fourier transform, gridding, preconditioner or solver step); both the CPU
oracle and the CUDA path take its outputs as plain arrays.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "ellipse_phantom", "coil_maps", "radial_golden_angle", "spiral_archimedean",
    "radial_3d_fibonacci", "complex_noise", "Workload", "workload", "batched_cases",
    "WORKLOADS",
]


def _pixel_coords(shape):
    """Centred pixel coordinates in FOV units: n_d / N_d with n_d in [-N_d/2, N_d/2)."""
    axes = [(np.arange(n) - n // 2) / n for n in shape]
    return np.meshgrid(*axes, indexing="ij")


def ellipse_phantom(shape, seed=0, n_ellipses=12, dtype=np.complex64):
    """Sum of random ellipses (ellipsoids in 3D) with a smooth global phase.

    Centres uniform in +-0.35 FOV, semi-axes uniform in [0.05, 0.35] FOV, random
    rotation, real amplitudes uniform in [0.1, 1.0] (additive), global phase
    exp(i*pi*0.2*(sum of coordinates)).
    """
    rng = np.random.default_rng(seed)
    grids = _pixel_coords(shape)
    d = len(shape)
    img = np.zeros(shape, dtype=np.float64)
    for _ in range(n_ellipses):
        centre = rng.uniform(-0.35, 0.35, size=d)
        axes = rng.uniform(0.05, 0.35, size=d)
        amp = rng.uniform(0.1, 1.0)
        if d == 2:
            a = rng.uniform(0, np.pi)
            rot = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
        else:
            # random rotation from a QR factorisation of a Gaussian matrix
            q, r = np.linalg.qr(rng.standard_normal((3, 3)))
            rot = q * np.sign(np.diag(r))
        rel = np.stack([g - c for g, c in zip(grids, centre)], axis=-1)
        loc = rel @ rot
        inside = np.sum((loc / axes) ** 2, axis=-1) <= 1.0
        img[inside] += amp
    phase = np.exp(1j * np.pi * 0.2 * sum(grids))
    return (img * phase).astype(dtype)


def coil_maps(shape, ncoils, seed=0, width=0.4, radius=0.6, dtype=np.complex64):
    """Gaussian-bump sensitivity maps normalised so sum_c |s_c[n]|^2 = 1 at every pixel.

    Coil c sits at angle 2*pi*c/C on a circle of radius ``radius`` FOV (2D) or on a
    Fibonacci sphere of that radius (3D); bump width ``width`` FOV; constant phase
    exp(i*pi*c/C).  ``seed`` only jitters the bump widths by +-5 % so that maps of
    different seeds differ.
    """
    rng = np.random.default_rng(seed)
    grids = _pixel_coords(shape)
    d = len(shape)
    maps = np.empty((ncoils,) + tuple(shape), dtype=np.complex128)
    for c in range(ncoils):
        if d == 2:
            ang = 2 * np.pi * c / ncoils
            centre = radius * np.array([np.cos(ang), np.sin(ang)])
        else:
            z = 1 - (2 * c + 1) / ncoils
            rho = math.sqrt(max(0.0, 1 - z * z))
            phi = c * math.pi * (3 - math.sqrt(5))
            centre = radius * np.array([z, rho * math.sin(phi), rho * math.cos(phi)])
        w = width * (1 + 0.05 * rng.uniform(-1, 1))
        r2 = sum((g - cc) ** 2 for g, cc in zip(grids, centre))
        maps[c] = np.exp(-r2 / (2 * w * w)) * np.exp(1j * np.pi * c / ncoils)
    sos = np.sqrt(np.sum(np.abs(maps) ** 2, axis=0))
    maps /= sos
    return maps.astype(dtype)


def radial_golden_angle(n_spokes, n_readout, kmax):
    """2D golden-angle radial: spoke s at angle s*pi*(sqrt(5)-1)/2, readout
    r_j = -kmax + j * (2*kmax/n_readout).  Returns float32 [M, 2] in cycles/FOV,
    ordered (k_y, k_x) to match row-major (y, x) image axes."""
    ga = np.pi * (math.sqrt(5) - 1) / 2
    ang = (np.arange(n_spokes) * ga) % np.pi
    r = -kmax + np.arange(n_readout) * (2.0 * kmax / n_readout)
    ky = np.sin(ang)[:, None] * r[None, :]
    kx = np.cos(ang)[:, None] * r[None, :]
    return np.stack([ky.ravel(), kx.ravel()], axis=-1).astype(np.float32)


def spiral_archimedean(n_interleaves, n_samples, kmax, undersampling=3.0):
    """Archimedean spiral, L interleaves, uniform time sampling t_j = j/n_samples.

    k(t) = kmax * t * exp(i(2*pi*T*t + 2*pi*l/L)); T = kmax/(undersampling*L) turns
    puts adjacent interleaves ``undersampling`` Nyquist units apart; uniform t gives a
    sample density decaying as 1/|k|.  Returns float32 [M, 2] (k_y, k_x)."""
    L = n_interleaves
    T = kmax / (undersampling * L)
    t = np.arange(n_samples) / n_samples
    out = []
    for l in range(L):
        ph = 2 * np.pi * T * t + 2 * np.pi * l / L
        r = kmax * t
        out.append(np.stack([r * np.sin(ph), r * np.cos(ph)], axis=-1))
    return np.concatenate(out, axis=0).astype(np.float32)


def radial_3d_fibonacci(n_spokes, n_readout, kmax):
    """3D centre-out radial: Fibonacci-sphere directions z_s = 1-(2s+1)/S,
    phi_s = s*pi*(3-sqrt(5)); r_j = kmax*j/n_readout.  float32 [M, 3] (k_z, k_y, k_x)."""
    s = np.arange(n_spokes)
    z = 1 - (2 * s + 1) / n_spokes
    rho = np.sqrt(np.maximum(0.0, 1 - z * z))
    phi = s * np.pi * (3 - math.sqrt(5))
    dirs = np.stack([z, rho * np.sin(phi), rho * np.cos(phi)], axis=-1)
    r = kmax * np.arange(n_readout) / n_readout
    return (dirs[:, None, :] * r[None, :, None]).reshape(-1, 3).astype(np.float32)


def complex_noise(shape, seed):
    """Unit-variance circular complex Gaussian noise (complex128)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


@dataclass
class Workload:
    """One synthetic reconstruction problem (inputs only)."""
    name: str
    img_shape: tuple
    ncoils: int
    oversamp: float
    width: int
    reg: str                 # "l2", "l1_wavelet" or "tv"
    lam_rel: float           # l2: lambda itself; l1: lambda / max|A^H y|
    iters: int
    wavelet_levels: int
    traj_kind: str
    traj_args: dict = field(default_factory=dict)
    seed: int = 0

    def traj(self):
        if self.traj_kind == "radial":
            return radial_golden_angle(**self.traj_args)
        if self.traj_kind == "spiral":
            return spiral_archimedean(**self.traj_args)
        if self.traj_kind == "radial3d":
            return radial_3d_fibonacci(**self.traj_args)
        raise ValueError(self.traj_kind)

    def phantom(self):
        return ellipse_phantom(self.img_shape, seed=self.seed)

    def maps(self):
        return coil_maps(self.img_shape, self.ncoils, seed=self.seed)

    def noise(self):
        m = self.traj().shape[0]
        return complex_noise((self.ncoils, m), seed=self.seed + 7)


WORKLOADS = {
    # 2D golden-angle radial, l2, 128^2, 4 coils, 64 x 256, alpha 2.0
    "radial2d_128": Workload("radial2d_128", (128, 128), 4, 2.0, 4, "l2", 1e-3, 30, 0,
                             "radial", dict(n_spokes=64, n_readout=256, kmax=64.0)),
    # 2D variable-density spiral, l1-wavelet, 256^2, 12 coils, 24 x 4096, alpha 1.25
    "spiral2d_256": Workload("spiral2d_256", (256, 256), 12, 1.25, 4, "l1_wavelet", 1e-3, 100, 4,
                             "spiral", dict(n_interleaves=24, n_samples=4096, kmax=128.0)),
    # 3D centre-out UTE radial, l1-wavelet, 192^3, 8 coils, 24000 x 256, alpha 1.25
    "ute3d_192": Workload("ute3d_192", (192, 192, 192), 8, 1.25, 4, "l1_wavelet", 1e-3, 30, 3,
                          "radial3d", dict(n_spokes=24000, n_readout=256, kmax=96.0)),
    # the same 3D trajectory family at a size whose grids (200^3 x 8 coils, 512 MB) still exceed
    # the L2 cache but keep a profiler capture within a few GB of device memory
    "ute3d_160": Workload("ute3d_160", (160, 160, 160), 8, 1.25, 4, "l1_wavelet", 1e-3, 30, 3,
                          "radial3d", dict(n_spokes=16000, n_readout=208, kmax=80.0)),
    # the 192^3 family's grid (240^3 passes, 8^3 tiles) with 2 coils and a quarter of the spokes:
    # 221 MB grids, above the L2 cache, and under 3 GB on the device for profiler captures
    "ute3d_192_c2": Workload("ute3d_192_c2", (192, 192, 192), 2, 1.25, 4, "l1_wavelet", 1e-3, 30, 3,
                             "radial3d", dict(n_spokes=6000, n_readout=256, kmax=96.0)),
    # differentiable unrolled solver: 2D spiral 256^2, 16 coils, 16 x 4096, l2 lambda 1e-2
    "spiral2d_256_unrolled": Workload("spiral2d_256_unrolled", (256, 256), 16, 1.25, 4, "l2", 1e-2, 10, 0,
                                      "spiral", dict(n_interleaves=16, n_samples=4096, kmax=128.0)),
}


def workload(name):
    return WORKLOADS[name]


def batched_cases(n_cases=64, base_seed=1000):
    """Descriptors of the uneven multi-case workload: image side uniform over
    multiples of 16 in [96, 320], coils uniform in [4, 32], spokes uniform in
    [32, 400] with 2*N readout samples, radial/spiral and l2/l1 by coin flips."""
    cases = []
    for i in range(n_cases):
        rng = np.random.default_rng(base_seed + i)
        n = int(rng.integers(6, 21)) * 16
        c = int(rng.integers(4, 33))
        spokes = int(rng.integers(32, 401))
        kind = "radial" if rng.uniform() < 0.5 else "spiral"
        reg = "l2" if rng.uniform() < 0.5 else "l1_wavelet"
        if kind == "radial":
            targs = dict(n_spokes=spokes, n_readout=2 * n, kmax=n / 2.0)
        else:
            targs = dict(n_interleaves=spokes, n_samples=2 * n, kmax=n / 2.0)
        cases.append(Workload(f"case{i}", (n, n), c, 1.25, 4, reg, 1e-3, 20,
                              4 if reg == "l1_wavelet" else 0, kind, targs, seed=base_seed + i))
    return cases
