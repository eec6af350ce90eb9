"""Pins of the oracle's trajectory derivatives and unrolled-PDHG gradients (no GPU):
central finite differences (step 1e-4 in cycles/FOV, skipping samples whose tap set would
change inside the step) and exact adjointness of the linear map y -> x_K."""
import numpy as np
import pytest

import synth
from oracle import gradients as og
from oracle import nufft as nf
from oracle import precond as opc
from oracle import solvers as osv


def _problem(shape=(16, 12), C=2, M=80, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    maps = rng.standard_normal((C,) + shape) + 1j * rng.standard_normal((C,) + shape)
    traj = np.stack([rng.uniform(-n / 2 + 1, n / 2 - 1, M) for n in shape], -1).astype(np.float64)
    return x, maps, traj


def _safe(traj, shape, h, alpha=1.25):
    g = nf.grid_shape(shape, alpha)
    t = traj * np.array([gg / n for gg, n in zip(g, shape)])
    fr = t - np.floor(t)
    return np.all((fr > 3 * h * 1.25) & (fr < 1 - 3 * h * 1.25), axis=1)


def test_kb_derivative_matches_fd():
    W, beta = 4, nf.kb_beta(4, 1.25)
    u = np.linspace(-1.99, 1.99, 101)
    h = 1e-6
    fd = (nf.kb_kernel(u + h, W, beta) - nf.kb_kernel(u - h, W, beta)) / (2 * h)
    assert np.allclose(og.kb_kernel_deriv(u, W, beta), fd, rtol=1e-6, atol=1e-6)
    # limit at the window edge
    assert abs(og.kb_kernel_deriv(np.array([2.0]), W, beta)[0] - (-2 * beta * beta * 2 / 16)) < 1e-12


def test_forward_traj_derivative_fd():
    x, maps, traj = _problem()
    h = 1e-4
    D = og.nufft_forward_dtraj(x, maps, traj)
    ok = _safe(traj, x.shape, h)
    assert ok.sum() > 40
    for d in range(2):
        tp, tm = traj.copy(), traj.copy()
        tp[:, d] += h
        tm[:, d] -= h
        fd = (nf.nufft_forward(x, maps, tp, 1.25, 4) - nf.nufft_forward(x, maps, tm, 1.25, 4)) / (2 * h)
        err = np.abs(D[:, ok, d] - fd[:, ok]).max() / np.abs(fd[:, ok]).max()
        assert err < 1e-5


def test_adjoint_traj_gradient_fd():
    x, maps, traj = _problem(seed=1)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((2, 80)) + 1j * rng.standard_normal((2, 80))
    gx = rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)
    h = 1e-4
    ok = _safe(traj, x.shape, h)
    G = og.traj_grad_adjoint(u, maps, traj, gx)
    Lf = lambda tr: float(np.real(np.vdot(gx, nf.nufft_adjoint(u, maps, tr, 1.25, 4))))
    for i in np.nonzero(ok)[0][:12]:
        for d in range(2):
            tp, tm = traj.copy(), traj.copy()
            tp[i, d] += h
            tm[i, d] -= h
            fd = (Lf(tp) - Lf(tm)) / (2 * h)
            assert abs(G[i, d] - fd) < 1e-4 * (abs(fd) + 1e-3)


@pytest.fixture(scope="module")
def unrolled():
    w = synth.Workload("u", (16, 16), 2, 1.25, 4, "l2", 1e-2, 6, 0, "spiral",
                       dict(n_interleaves=4, n_samples=40, kmax=8.0))
    x0, maps, traj = w.phantom().astype(np.complex128), w.maps().astype(np.complex128), w.traj().astype(np.float64)
    rng = np.random.default_rng(2)
    y = nf.nufft_forward(x0, maps, traj) + 0.05 * (rng.standard_normal((2, traj.shape[0])) + 0)
    p = opc.mc_precond_fast(maps, traj.astype(np.float32), 1.25, 4)
    A = lambda v: nf.nufft_forward(v, maps, traj)
    AH = lambda u: nf.nufft_adjoint(u, maps, traj)
    L, _ = osv.power_method(A, AH, p, x0.shape)
    return dict(y=y, maps=maps, traj=traj, p=p, L=L, lam=1e-2, iters=6, shape=x0.shape)


def _loss(xK, c):
    return float(np.real(np.vdot(c, xK)))    # real, linear loss: dL/dx = c


def test_unrolled_matches_pdhg(unrolled):
    u = unrolled
    xK, _ = og.unrolled_pdhg_l2(u["y"], u["maps"], u["traj"], u["p"], u["lam"], u["iters"], u["L"])
    A = lambda v: nf.nufft_forward(v, u["maps"], u["traj"])
    AH = lambda r: nf.nufft_adjoint(r, u["maps"], u["traj"])
    xr, _, _, _ = osv.pdhg(A, AH, u["y"], u["p"], u["shape"], "l2", u["lam"], u["iters"], u["L"])
    assert np.abs(xK - xr).max() < 1e-12 * np.abs(xr).max()


def test_unrolled_grad_y_is_exact_adjoint(unrolled):
    """y -> x_K is linear for l2: <g_y, dy> must equal <c, x_K(dy)> exactly."""
    u = unrolled
    rng = np.random.default_rng(3)
    c = rng.standard_normal(u["shape"]) + 1j * rng.standard_normal(u["shape"])
    xK, tape = og.unrolled_pdhg_l2(u["y"], u["maps"], u["traj"], u["p"], u["lam"], u["iters"], u["L"])
    gy, _, _ = og.unrolled_pdhg_l2_grad(c, u["y"], u["maps"], u["traj"], u["p"], u["lam"], u["iters"], u["L"],
                                        tape, want_traj=False)
    dy = rng.standard_normal(u["y"].shape) + 1j * rng.standard_normal(u["y"].shape)
    xd, _ = og.unrolled_pdhg_l2(dy, u["maps"], u["traj"], u["p"], u["lam"], u["iters"], u["L"])
    assert abs(float(np.real(np.vdot(gy, dy))) - _loss(xd, c)) < 1e-10 * abs(_loss(xd, c))


def test_unrolled_grad_lambda_and_traj_fd(unrolled):
    u = unrolled
    rng = np.random.default_rng(4)
    c = rng.standard_normal(u["shape"]) + 1j * rng.standard_normal(u["shape"])
    run = lambda lam, tr: _loss(og.unrolled_pdhg_l2(u["y"], u["maps"], tr, u["p"], lam, u["iters"], u["L"])[0], c)
    xK, tape = og.unrolled_pdhg_l2(u["y"], u["maps"], u["traj"], u["p"], u["lam"], u["iters"], u["L"])
    _, glam, gf = og.unrolled_pdhg_l2_grad(c, u["y"], u["maps"], u["traj"], u["p"], u["lam"], u["iters"], u["L"], tape)
    h = 1e-6
    fd = (run(u["lam"] + h, u["traj"]) - run(u["lam"] - h, u["traj"])) / (2 * h)
    assert abs(glam - fd) < 1e-6 * abs(fd)
    h = 1e-4
    ok = _safe(u["traj"], u["shape"], h)
    for i in np.nonzero(ok)[0][::17][:8]:
        d = i % 2
        tp, tm = u["traj"].copy(), u["traj"].copy()
        tp[i, d] += h
        tm[i, d] -= h
        fdt = (run(u["lam"], tp) - run(u["lam"], tm)) / (2 * h)
        assert abs(gf[i, d] - fdt) < 2e-4 * (abs(fdt) + 1e-2 * np.abs(gf).max())
