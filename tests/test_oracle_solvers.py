"""Pins of the oracle's power method and preconditioned PDHG (no GPU).  Sec. 4.1, Sec. 6."""
import numpy as np
import pytest

import synth
from oracle import nufft as nf
from oracle import precond as pc
from oracle import solvers as sv


@pytest.fixture(scope="module")
def prob():
    rng = np.random.default_rng(3)
    shape, C = (16, 16), 3
    x0 = synth.ellipse_phantom(shape, seed=1).astype(np.complex128)
    maps = synth.coil_maps(shape, C, seed=1).astype(np.complex128)
    traj = synth.radial_golden_angle(12, 32, 8.0)
    M = traj.shape[0]
    A = nf.sense_matrix(maps, traj)
    Af = lambda v: (A @ v.ravel()).reshape(C, M)
    AHf = lambda u: (A.conj().T @ u.ravel()).reshape(shape)
    y = Af(x0) + 0.01 * (rng.standard_normal((C, M)) + 1j * rng.standard_normal((C, M)))
    p = pc.precond_bruteforce(A).reshape(C, M)
    return dict(A=A, Af=Af, AHf=AHf, y=y, p=p, shape=shape)


def test_power_method_matches_eigvalsh(prob):
    A, p = prob["A"], prob["p"]
    P = np.sqrt(p.ravel())
    ev = np.linalg.eigvalsh((P[:, None] * A) @ (A.conj().T * P[None, :])).max()
    L, _ = sv.power_method(prob["Af"], prob["AHf"], p, prob["shape"], iters=300)
    assert abs(L - ev) < 1e-8 * ev
    L30, _ = sv.power_method(prob["Af"], prob["AHf"], p, prob["shape"], iters=30)
    assert L30 <= ev * (1 + 1e-12) and L30 > 0.9 * ev


def test_schedule_invariant():
    sched = sv.pdhg_schedule(50, 3.7, 0.21)
    st = [s * t for s, t, _ in sched]
    assert np.allclose(st, 1 / 3.7, rtol=1e-14, atol=0)
    assert sched[0][0] == 1.0 and abs(sched[0][1] - 1 / 3.7) < 1e-15
    for (s0, _, th), (s1, _, _) in zip(sched, sched[1:]):
        assert abs(th - 1 / (1 + 2 * s0 * 0.21)) < 1e-15 and abs(s1 - th * s0) < 1e-15


def test_pdhg_l2_fixed_point_is_cg_solution(prob):
    """(x*, u* = A x* - y) with -A^H u* = lam x* is a fixed point of the iteration (sign pin)."""
    lam = 1e-2
    xs = sv.cg_l2(prob["Af"], prob["AHf"], prob["y"], lam, prob["shape"])
    us = prob["Af"](xs) - prob["y"]
    assert np.linalg.norm(-prob["AHf"](us) - lam * xs) < 1e-8 * np.linalg.norm(lam * xs)
    x, u, _, _ = sv.pdhg(prob["Af"], prob["AHf"], prob["y"], prob["p"], prob["shape"], "l2", lam, 5,
                         1.5, state=(xs, xs, us, 7))
    assert np.linalg.norm(x - xs) < 1e-9 * np.linalg.norm(xs)
    assert np.linalg.norm(u - us) < 1e-9 * np.linalg.norm(us)


def test_pdhg_l2_converges_to_cg(prob):
    lam = 1e-2
    xs = sv.cg_l2(prob["Af"], prob["AHf"], prob["y"], lam, prob["shape"])
    L, _ = sv.power_method(prob["Af"], prob["AHf"], prob["p"], prob["shape"])
    errs = []
    for it in (30, 300, 1000):
        x, _, _, _ = sv.pdhg(prob["Af"], prob["AHf"], prob["y"], prob["p"], prob["shape"], "l2", lam, it, L)
        errs.append(np.linalg.norm(x - xs) / np.linalg.norm(xs))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 5e-5


def test_preconditioning_speeds_up(prob):
    """Sec. 6 claim, qualitatively: after 30 iterations MC-preconditioned PDHG is closer to the
    optimum than unpreconditioned PDHG."""
    lam = 1e-2
    xs = sv.cg_l2(prob["Af"], prob["AHf"], prob["y"], lam, prob["shape"])
    ones = np.ones_like(prob["p"])
    res = []
    for p in (prob["p"], ones):
        L, _ = sv.power_method(prob["Af"], prob["AHf"], p, prob["shape"])
        x, _, _, _ = sv.pdhg(prob["Af"], prob["AHf"], prob["y"], p, prob["shape"], "l2", lam, 30, L)
        res.append(np.linalg.norm(x - xs))
    assert res[0] < res[1]


def test_pdhg_l1_matches_fista(prob):
    lam = 1e-3
    L, _ = sv.power_method(prob["Af"], prob["AHf"], prob["p"], prob["shape"])
    x, u, _, objs = sv.pdhg(prob["Af"], prob["AHf"], prob["y"], prob["p"], prob["shape"], "l1_wavelet",
                            lam, 1500, L, levels=2, trace=True)
    xf = sv.fista_l1(prob["Af"], prob["AHf"], prob["y"], lam, prob["shape"], 2, iters=3000)
    ff = sv.objective(prob["Af"], xf, prob["y"], "l1_wavelet", lam, 2)
    assert abs(objs[-1] - ff) < 1e-5 * ff
    # fixed point of the l1 prox-gradient map at the PDHG solution
    t = 0.5 / 1.5
    from oracle import wavelet as wv
    g = wv.prox_l1_wavelet(x - t * prob["AHf"](prob["Af"](x) - prob["y"]), t * lam, 2)
    assert np.linalg.norm(g - x) < 1e-3 * np.linalg.norm(x)
