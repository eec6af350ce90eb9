"""Helpers shared by the GPU parity tests: seeded problems and relative errors.

Inputs come from ``synth`` (shared seeded generators); expected values come only from
``oracle`` (float64 CPU).  The CUDA path is reached through ``paper_1902_09657_gb300.api``
(ctypes over the C ABI).
"""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import nufft as onf

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_09657_gb300 import _build
    _build.build()


MEASURED = []


def rel(a, b, what=""):
    """Relative l2 error ||a - b|| / ||b||; every value is kept with the test that measured it and
    written to $KPDHG_PARITY_LOG (JSON lines) when that variable is set."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    e = float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
    test = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    MEASURED.append((test, what, e))
    path = os.environ.get("KPDHG_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": test, "what": what, "rel_err": e}) + "\n")
    return e


def rounded(t):
    """Values of a half-storage tensor [..., 2] (or complex64) as complex128 on the host: the
    exact inputs the GPU computed with, for arithmetic parity against the oracle."""
    if t.dtype == torch.complex64:
        return t.cpu().numpy().astype(np.complex128)
    f = t.float().cpu().numpy().astype(np.float64)
    return f[..., 0] + 1j * f[..., 1]


def random_problem(shape, C, M, seed, edge=False):
    """Random image, random maps and uniformly random coordinates in [-N/2, N/2)."""
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    maps = (rng.standard_normal((C,) + shape) + 1j * rng.standard_normal((C,) + shape)).astype(np.complex64)
    traj = np.stack([rng.uniform(-n / 2, n / 2, M) for n in shape], -1).astype(np.float32)
    if edge:
        # boundary and on-grid coordinates exercise the float32 first-tap decision and wrap-around
        k = min(M, 8)
        traj[:k] = np.array([[(-1) ** j * n / 2 for n in shape] for j in range(k)], dtype=np.float32)
        traj[k:2 * k] = np.round(traj[k:2 * k])
    return x, maps, traj


def workload_problem(name):
    w = synth.workload(name)
    traj = w.traj()
    x = w.phantom()
    maps = w.maps()
    return w, x, maps, traj


def simulate(w, x, maps, traj):
    """Measurements from the oracle's accurate NUFFT (alpha 2, W 8) plus 1 % noise."""
    return onf.simulate_kspace(x.astype(np.complex128), maps.astype(np.complex128), traj, w.noise()).astype(np.complex64)


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def make_plan(x_shape, C, M, oversamp=1.25, levels=0):
    from paper_1902_09657_gb300.api import Plan
    return Plan(x_shape, C, M, oversamp=oversamp, wavelet_levels=levels)
