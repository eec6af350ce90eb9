"""Pins of the oracle's Daubechies-4 wavelet and l1 prox (no GPU).  Sec. 2 (W unitary), Sec. 6 (db4)."""
import math
import os

import numpy as np

from oracle import wavelet as wv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    out = {}
    for line in open(os.path.join(GOLDEN, "db4_properties.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        out[k] = float(v)
    return out


def test_filter_properties():
    g = _golden()
    h = wv.daubechies_filter(4)
    assert len(h) == g["taps"]
    assert abs(h.sum() - g["sum"]) < 1e-14
    assert abs((h ** 2).sum() - g["energy"]) < 1e-14
    for k in (1, 2, 3):
        assert abs(sum(h[n] * h[n + 2 * k] for n in range(8 - 2 * k))) < 1e-14
    for m in range(int(g["vanishing_moments"])):
        assert abs(sum((-1) ** n * n ** m * h[n] for n in range(8))) < 1e-11
    # the 5th moment does not vanish (exactly 4 vanishing moments)
    assert abs(sum((-1) ** n * n ** 4 * h[n] for n in range(8))) > 1e-3


def test_filter_is_minimum_phase():
    """Extremal phase: all zeros of H(z) on or inside the unit circle, so energy is front-loaded."""
    h = wv.daubechies_filter(4)
    zeros = np.roots(h)
    assert np.all(np.abs(zeros) < 1 + 1e-3)
    assert (h[:4] ** 2).sum() > 0.9


def test_haar_special_case_by_hand():
    """p = 1 gives the Haar filter [1, 1]/sqrt(2); one level on [a, b, c, d] by hand."""
    h = wv.daubechies_filter(1)
    assert np.allclose(h, [1 / math.sqrt(2)] * 2)
    x = np.array([1.0, 3.0, 2.0, 6.0])
    c = wv.dwt_level_axis(x, 0, h)
    s = 1 / math.sqrt(2)
    # g = [h1, -h0] = [s, -s]
    assert np.allclose(c, [4 * s, 8 * s, -2 * s, -4 * s])


def test_perfect_reconstruction_and_unitarity_2d_3d():
    rng = np.random.default_rng(0)
    for shape, lev in (((32, 16), 3), ((16, 8, 8), 2), ((64, 64), 4)):
        x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        c = wv.dwt(x, lev)
        assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
        assert np.abs(wv.idwt(c, lev) - x).max() < 1e-12
        y = rng.standard_normal(shape) + 0j
        assert abs(np.vdot(wv.dwt(y, lev), c) - np.vdot(y, x)) < 1e-10


def test_cubic_has_no_interior_detail():
    """4 vanishing moments: a cubic polynomial gives zero detail away from the periodic seam."""
    n = np.arange(64, dtype=float)
    x = 0.3 * n ** 3 - 2 * n ** 2 + n - 5
    c = wv.dwt_level_axis(x, 0, wv.daubechies_filter(4))
    d = c[32:]
    assert np.abs(d[:28]).max() < 1e-8 * np.abs(x).max()
    assert np.abs(d[28:]).max() > 1.0   # the seam (wrap-around) is not polynomial


def test_soft_threshold():
    c = np.array([0.0, 3 + 4j, 0.5, -2.0])
    s = wv.soft_threshold(c, 1.0)
    assert np.allclose(s, [0.0, (3 + 4j) * 0.8, 0.0, -1.0])


def test_prox_l1_wavelet_is_minimiser():
    """prox_{t||W.||_1}(z) minimises ||x - z||^2/2 + t||Wx||_1: random perturbations do worse."""
    rng = np.random.default_rng(1)
    z = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    t = 0.4
    x = wv.prox_l1_wavelet(z, t, 2)
    f = lambda v: 0.5 * np.linalg.norm(v - z) ** 2 + t * np.abs(wv.dwt(v, 2)).sum()
    f0 = f(x)
    for _ in range(20):
        d = 1e-3 * (rng.standard_normal(z.shape) + 1j * rng.standard_normal(z.shape))
        assert f(x + d) >= f0 - 1e-12
