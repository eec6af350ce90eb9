"""Pins of the oracle's objective F(x) = 1/2 ||A x - y||^2 + g(x) (Eq. obj) against values fixed
by the mathematics rather than by the objective's own formula (no GPU).

* l1-wavelet term, constant image x = c: an orthonormal periodised filter bank with
  sum_n h[n] = sqrt(2) and sum_n g[n] = 0 maps a constant onto the coarsest approximation band
  only; after L levels in d dimensions that band holds (n/2^L)^d coefficients, each c 2^{dL/2},
  so ||W x||_1 = |c| n^d / 2^{dL/2}.
* l1-wavelet term, checkerboard x[j] = prod_d (-1)^{j_d}: the low-pass response at pi is zero
  (H(pi) = 0, four vanishing moments) and the high-pass one is sum_n (-1)^n g[n] = sqrt(2), so
  the first level puts 2^{d/2} into every coefficient of the all-high band and nothing elsewhere:
  ||W x||_1 = n^d 2^{d/2} / 2^d, independent of the number of levels.
* data term: y = A x - 3 e_0 gives 1/2 ||A x - y||^2 = 4.5 exactly.
* l2 at its optimum: min_x 1/2 ||A x - y||^2 + lambda/2 ||x||^2 = 1/2 y^H (I - A (A^H A + lambda I)^{-1} A^H) y
  (completing the square), evaluated with a dense solve.
* TV: ||G x||_1 of the checkerboard is 2 d n^d (every periodic difference has magnitude 2),
  of a constant 0.

Each plausible slip (sum |x| instead of sum |W x|, a dropped approximation band, a dropped
1/2 on either term, lambda instead of lambda/2 on the l2 term) is planted in a copy of the
objective below and must break at least one pin.
"""
import math

import numpy as np
import pytest

import synth
from oracle import nufft as nf
from oracle import solvers as sv
from oracle import wavelet as wv


@pytest.fixture(scope="module")
def tiny():
    shape, C = (16, 16), 2
    maps = synth.coil_maps(shape, C, seed=3).astype(np.complex128)
    traj = synth.radial_golden_angle(10, 24, 8.0)
    A = nf.sense_matrix(maps, traj)
    M = traj.shape[0]
    Af = lambda v: (A @ v.ravel()).reshape(C, M)
    return dict(shape=shape, A=A, Af=Af, C=C, M=M)


def _pins(obj, t):
    """True when `obj(A, x, y, reg, lam, levels)` meets every closed form above."""
    shape, Af = t["shape"], t["Af"]
    n = shape[0]
    d = len(shape)
    ok = True
    lam = 0.37
    # constant image, y = A x: only the coarsest approximation band is non-zero
    for L in (1, 2, 3):
        c = 0.8 - 0.6j
        x = np.full(shape, c)
        want = lam * abs(c) * n ** d / 2 ** (d * L / 2)
        ok &= abs(obj(Af, x, Af(x), "l1_wavelet", lam, L) - want) < 1e-10 * want
    # checkerboard: only the first level's all-high band, 2^{d/2} per coefficient
    j = np.indices(shape).sum(axis=0)
    x = (-1.0) ** j + 0j
    want = lam * n ** d * 2 ** (d / 2) / 2 ** d
    for L in (1, 3):
        ok &= abs(obj(Af, x, Af(x), "l1_wavelet", lam, L) - want) < 1e-10 * want
    # data term with a planted residual of norm 3
    rng = np.random.default_rng(5)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    r = np.zeros((t["C"], t["M"]), dtype=np.complex128)
    r[0, 0] = 3.0
    for reg in ("l2", "l1_wavelet"):
        ok &= abs(obj(Af, x, Af(x) - r, reg, 0.0, 2) - 4.5) < 1e-10
    # l2 objective at its minimiser: completing the square
    A = t["A"]
    y = (rng.standard_normal((t["C"], t["M"])) + 1j * rng.standard_normal((t["C"], t["M"]))).ravel()
    lam2 = 0.05
    H = A.conj().T @ A + lam2 * np.eye(A.shape[1])
    xs = np.linalg.solve(H, A.conj().T @ y)
    want = 0.5 * float(np.real(np.vdot(y, y - A @ np.linalg.solve(H, A.conj().T @ y))))
    got = obj(Af, xs.reshape(shape), y.reshape(t["C"], t["M"]), "l2", lam2, 0)
    ok &= abs(got - want) < 1e-9 * abs(want)
    return bool(ok)


def test_objective_meets_closed_forms(tiny):
    assert _pins(sv.objective, tiny)


def _mutant(kind):
    def obj(A, x, y, reg, lam, levels=0):
        r = A(x) - y
        half = 1.0 if kind == "no_half_data" else 0.5
        f = half * float(np.vdot(r, r).real)
        if reg == "l2":
            f += (1.0 if kind == "l2_weight" else 0.5) * lam * float(np.vdot(x, x).real)
        elif kind == "abs_x":
            f += lam * float(np.sum(np.abs(x)))
        elif kind == "no_approx":
            cw = wv.dwt(x, levels)
            blk = tuple(slice(0, s >> levels) for s in x.shape)
            cw[blk] = 0
            f += lam * float(np.sum(np.abs(cw)))
        elif kind == "no_details":
            cw = wv.dwt(x, levels)
            blk = tuple(slice(0, s >> levels) for s in x.shape)
            f += lam * float(np.sum(np.abs(cw[blk])))
        else:
            f += lam * float(np.sum(np.abs(wv.dwt(x, levels))))
        return f
    return obj


@pytest.mark.parametrize("kind", ["abs_x", "no_approx", "no_details", "no_half_data", "l2_weight"])
def test_planted_objective_slips_break_a_pin(tiny, kind):
    assert not _pins(_mutant(kind), tiny)


def test_tv_objective_closed_forms(tiny):
    shape, Af = tiny["shape"], tiny["Af"]
    n, d = shape[0], len(shape)
    lam = 0.21
    j = np.indices(shape).sum(axis=0)
    x = (-1.0) ** j * (0.6 + 0.8j)
    assert abs(sv.objective_tv(Af, x, Af(x), lam) - lam * 2 * d * n ** d) < 1e-10 * lam * n ** d
    x = np.full(shape, 2.0 - 1.0j)
    assert sv.objective_tv(Af, x, Af(x), lam) == 0.0
    r = np.zeros((tiny["C"], tiny["M"]), dtype=np.complex128)
    r[1, 3] = 3.0
    assert abs(sv.objective_tv(Af, x, Af(x) - r, lam) - 4.5) < 1e-10
