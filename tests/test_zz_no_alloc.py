"""The allocation-free adjoint (kp_sense_adjoint_noalloc) against the plan-based kp_sense_adjoint
and against the float64 oracle's adjoint.

The allocation-free entry point exists for callers that reserve all device memory up front
and cannot let a library allocate in the middle of a reconstruction.  It keeps its work space
in one fixed device array shared by every call, so this test calls it twice in a row with
different data (the second call must not see the first call's grid), in 2D and 3D, and checks
that an oversize problem is refused.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from oracle import nufft as onf
from tests.gpu_util import need_gpu, rel, random_problem, to_dev, make_plan

pytestmark = pytest.mark.gpu


def _params(shape, C, M, alpha=1.25):
    from paper_1902_09657_gb300 import _lib
    prm = _lib.KpParams()
    prm.ndim = len(shape)
    for d, n in enumerate(shape):
        prm.img[d] = n
    prm.ncoils, prm.nsamples, prm.oversamp, prm.kernel_width, prm.wavelet_levels = C, M, alpha, 4, 0
    return prm


def _noalloc(prm, traj_d, maps_d, y_d, x_d):
    import torch
    from paper_1902_09657_gb300 import _lib
    lib = _lib.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    s = lib.kp_sense_adjoint_noalloc(ctypes.byref(prm), ctypes.c_void_p(traj_d.data_ptr()),
                                     ctypes.c_void_p(maps_d.data_ptr()), ctypes.c_void_p(y_d.data_ptr()),
                                     ctypes.c_void_p(x_d.data_ptr()), st)
    return s


@pytest.mark.parametrize("shape,C,M", [((64, 48), 6, 3000), ((16, 20, 12), 2, 900)])
def test_noalloc_adjoint_matches_plan_adjoint_twice(shape, C, M):
    need_gpu()
    import torch
    from paper_1902_09657_gb300 import _lib
    _, maps, traj = random_problem(shape, C, M, 11, edge=True)
    plan = make_plan(shape, C, M)
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    prm = _params(shape, C, M)
    traj_d, maps_d = to_dev(traj), to_dev(maps)
    for call in range(2):
        rng = np.random.default_rng(100 + call)
        y = (rng.standard_normal((C, M)) + 1j * rng.standard_normal((C, M))).astype(np.complex64)
        y_d = to_dev(y)
        ref = plan.sense_adjoint(y_d).cpu().numpy()
        x_d = torch.empty(shape, dtype=torch.complex64, device="cuda")
        assert _noalloc(prm, traj_d, maps_d, y_d, x_d) == _lib.KP_OK
        torch.cuda.synchronize()
        got = x_d.cpu().numpy()
        assert rel(got, ref, f"call {call} vs plan adjoint") < 1e-5
        x_ref = onf.nufft_adjoint(y.astype(np.complex128), maps.astype(np.complex128), traj, 1.25, 4)
        assert rel(got, x_ref, f"call {call} vs oracle") < 1e-5


def test_noalloc_rejects_oversize_problem():
    need_gpu()
    import torch
    from paper_1902_09657_gb300 import _lib
    shape, C, M = (256, 256), 12, 16
    prm = _params(shape, C, M)
    d = torch.zeros(16, dtype=torch.complex64, device="cuda")
    s = _noalloc(prm, d, d, d, d)
    assert s == _lib.KP_EINVAL
    assert b"too large" in _lib.load().kp_last_error()
