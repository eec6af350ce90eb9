"""Cases run by the bounds-checked library test (tests/test_gpu_checked.py).

``run_cases()`` drives the library through the public API on small 2D and 3D problems that
reach every instrumented kernel: bin-sort, forward and adjoint NUFFT (the one-phase 2D
spreading and the two-phase 3D spreading with its own phase and gather, the interpolation,
the library's own 3D FFT passes), the MC preconditioner, the power method and PDHG with the
fused primal step (l1-wavelet and l2).  Run as a script (``python -m tests.checked_cases
OUT.npz``, with KPDHG_CHECKED=1 for the checked build; ``--workload NAME`` runs one whole
reconstruction of a named workload at full size instead) it saves the results and prints the
library's bounds report as one JSON line.
"""
import json
import os
import sys

import numpy as np

import synth


def _problem(shape, C, traj, seed):
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    maps = (rng.standard_normal((C,) + shape) + 1j * rng.standard_normal((C,) + shape)).astype(np.complex64)
    u = (rng.standard_normal((C, traj.shape[0])) + 1j * rng.standard_normal((C, traj.shape[0]))).astype(np.complex64)
    return x, maps, u


def run_cases():
    import torch
    from paper_1902_09657_gb300.api import Plan
    out = {}
    cases = [
        # 2D spiral, one-phase spreading (variant 6), cuFFT
        ("spiral2d", (64, 64), 4, 3, synth.spiral_archimedean(n_interleaves=8, n_samples=1024, kmax=32.0), "6", "256"),
        # 3D centre-out radial, two-phase spreading (variant 10, 4096-sample own items), own FFT passes (60^3)
        ("radial3d", (48, 48, 48), 3, 2, synth.radial_3d_fibonacci(n_spokes=400, n_readout=48, kmax=24.0), "10", "4096"),
    ]
    for name, shape, C, levels, traj, variant, chunk in cases:
        os.environ["KPDHG_SPREAD_VARIANT"] = variant
        os.environ["KPDHG_SPREAD_CHUNK"] = chunk
        x, maps, u = _problem(shape, C, traj, len(shape))
        M = traj.shape[0]
        plan = Plan(shape, C, M, wavelet_levels=levels)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        plan.set_trajectory(dev(traj)).set_maps(dev(maps))
        y = plan.sense_forward(dev(x))
        out[f"{name}_forward"] = y.cpu().numpy()
        out[f"{name}_adjoint"] = plan.sense_adjoint(dev(u)).cpu().numpy()
        p = plan.make_preconditioner(True)
        out[f"{name}_precond"] = p.cpu().numpy()
        lmax = plan.max_eig(p, iters=10)
        out[f"{name}_lmax"] = np.array([lmax])
        lam = 1e-3 * float(plan.sense_adjoint(y).abs().max())
        xl1, _, _ = plan.pdhg_solve(y, p, "l1_wavelet", lam, 8, lmax=lmax)
        out[f"{name}_pdhg_l1"] = xl1.cpu().numpy()
        xl2, _, _ = plan.pdhg_solve(y, p, "l2", 1e-3, 8, lmax=lmax)
        out[f"{name}_pdhg_l2"] = xl2.cpu().numpy()
        plan.close()
    os.environ.pop("KPDHG_SPREAD_VARIANT", None)
    os.environ.pop("KPDHG_SPREAD_CHUNK", None)
    return out


def run_workload(name):
    """One whole reconstruction of a named workload (bin-sort, MC preconditioner, 30 power
    iterations, the workload's PDHG iterations) at its full size, with the storage types the
    bench uses; returns the image."""
    import torch
    from paper_1902_09657_gb300.api import Plan, to_storage
    w = synth.workload(name)
    traj = w.traj()
    plan = Plan(w.img_shape, w.ncoils, traj.shape[0], oversamp=w.oversamp, wavelet_levels=w.wavelet_levels)
    maps = torch.from_numpy(w.maps()).cuda()
    maps_st = to_storage(maps, "fp16") if len(w.img_shape) == 3 else maps
    plan.set_trajectory(torch.from_numpy(traj).cuda()).set_maps(maps_st)
    y = plan.sense_forward(torch.from_numpy(w.phantom()).cuda())
    lam = 1e-3 * float(plan.sense_adjoint(y).abs().max())
    x, _, _ = plan.pdhg_solve(y, None, w.reg, lam, w.iters)
    out = x.cpu().numpy()
    plan.close()
    return out


def main(argv):
    from paper_1902_09657_gb300.api import bounds_report
    if len(argv) > 2 and argv[2] == "--workload":
        res = {"x": run_workload(argv[3])}
    else:
        res = run_cases()
    np.savez(argv[1], **res)
    print(json.dumps(bounds_report()), flush=True)


if __name__ == "__main__":
    main(sys.argv)
