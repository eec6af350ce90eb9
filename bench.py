#!/usr/bin/env python
"""Benchmark of k-space-preconditioned PDHG (Ong, Uecker & Lustig, arXiv 1902.09657) on GB300.

One timed step = one whole reconstruction of the 3D centre-out UTE radial l1-wavelet workload
(192^3 image, 8 coils with coil maps stored in FP16, 24,000 Fibonacci-sphere spokes x 256
samples, oversampling 1.25, KB width 4, Daubechies-4 with 3 levels, lambda = 1e-3 max|A^H y|):
trajectory binning, coil maps, multi-channel preconditioner, 30 power iterations, 30 PDHG
iterations.  All inputs are synthetic (seeded ellipsoid phantom, Gaussian-bump coil maps,
Fibonacci-sphere trajectory, Gaussian noise).  The same JSON line carries the 2D spiral
(256^2 x 12 coils, 100 l1 iterations) and 2D radial (128^2 x 4 coils, 30 l2 iterations)
reconstructions, the 64-case batch, the unrolled gradient and the mixed-precision forms.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank reconstructs its own
replica of the workload (independent problems, weak scaling); ranks only meet in the
barriers and the max-over-ranks of the timing.  --impl reference times the float64 CPU
oracle on a bounded sample of the same workload and extrapolates the whole reconstruction.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOAD = "ute3d_192"
# (maps storage, measurement storage) of each timed workload: the 3D workload keeps its coil
# maps in FP16 (FP32 arithmetic); the others are plain complex64
STORAGE = {"ute3d_192": ("fp16", "c64"), "ute3d_160": ("fp16", "c64"), "ute3d_192_c2": ("fp16", "c64")}


def storage_of(w):
    return STORAGE.get(w.name, ("c64", "c64"))


def metric_name(w):
    reg = "l1-wavelet" if w.reg == "l1_wavelet" else "l2"
    return (f"PDHG iterations/s, whole reconstruction (bin-sort + MC preconditioner + 30 power its + "
            f"{w.iters} {reg} PDHG its)")


def lambda_for(w, ahy_max=None):
    """l2: lambda itself; l1: lam_rel * max|A^H y|."""
    return w.lam_rel * ahy_max if w.reg == "l1_wavelet" else w.lam_rel


def parse():
    return parse_args_list(None)


def parse_args_list(argv):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.WORKLOADS),
                    help="timed workload (default: the 3D UTE l1-wavelet reconstruction)")
    ap.add_argument("--no-extras", action="store_true", help="skip roofline/e2e/time-to-accuracy extras")
    ap.add_argument("--no-side-workloads", action="store_true",
                    help="skip the 2D, 64-case batch and unrolled-gradient side measurements")
    return ap.parse_args(argv)


def grid_points(w):
    G = 1
    for n in w.img_shape:
        g = math.ceil(w.oversamp * n - 1e-9)
        G *= g + (g % 2)
    return G


def n_samples(w):
    ta = w.traj_args
    return ta["n_interleaves"] * ta["n_samples"] if w.traj_kind == "spiral" else ta["n_spokes"] * ta["n_readout"]


def workload_config(w):
    ta = w.traj_args
    if w.traj_kind == "spiral":
        traj = f"{ta['n_interleaves']}x{ta['n_samples']} spiral samples"
    else:
        traj = f"{ta['n_spokes']}x{ta['n_readout']} {w.traj_kind} samples"
    shape = "x".join(str(n) for n in w.img_shape)
    reg = ("l1 lambda=1e-3*max|A^H y|, db4 %d levels" % w.wavelet_levels if w.reg == "l1_wavelet"
           else "l2 lambda=%g" % w.lam_rel)
    ms, ys = storage_of(w)
    grid_mb = w.ncoils * grid_points(w) * 8 / 1e6
    return {
        "workload": f"{w.name}: {shape} image, {w.ncoils} coils, {traj}, alpha {w.oversamp}, KB W{w.width}, "
                    f"{reg}, {w.iters} iterations, maps {ms}, y {ys}",
        "image": list(w.img_shape), "coils": w.ncoils, "samples": int(n_samples(w)),
        "iters": w.iters, "power_iters": 30, "preconditioner": "multi-channel",
        "maps_storage": ms, "y_storage": ys,
        "l2_between_steps": f"flushed (256 MiB write); per-coil grids total {grid_mb:.0f} MB",
    }


# ----------------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- multi-rank
def max_over_ranks(total_ms, world, device="cpu"):
    """Slowest rank's timed-region length (every rank runs its own replica: weak scaling)."""
    if world == 1:
        return float(total_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, steps, iters, total_ms):
    """PDHG iterations per second summed over all ranks' replicas, timed by the slowest."""
    return world * steps * iters / (total_ms / 1e3)


# ----------------------------------------------------------------------------- oracle
def _nlogn(n):
    return n * math.log2(max(n, 2))


def oracle_inputs(w):
    """Float64 oracle inputs of the workload (phantom, maps rounded to their storage, trajectory)."""
    x = w.phantom().astype(np.complex128)
    maps = w.maps()
    if storage_of(w)[0] == "fp16":
        maps = maps.view(np.float32).astype(np.float16).astype(np.float32).view(np.complex64)
    return x, maps.astype(np.complex128), w.traj()


def oracle_calibrate(w, x, maps, traj, m1):
    """Once per run: the oracle's prox on the full image, one FFT of a single coil's oversampled
    grid (the library step inside every oracle NUFFT), and its forward + adjoint NUFFT on the
    first m1 samples with one and with two coils, which separates the gridding cost per call
    (tap tables) from the cost per coil.  Seconds."""
    from oracle import nufft as onf, solvers as osv
    gshape = onf.grid_shape(w.img_shape, w.oversamp)
    grid = np.zeros(gshape, dtype=np.complex128)
    grid[tuple(slice(0, n) for n in w.img_shape)] = x
    t0 = time.perf_counter()
    np.fft.fftn(grid)
    t_fft = time.perf_counter() - t0
    del grid
    prox = osv.make_prox(w.reg, 1e-3, w.wavelet_levels)
    t0 = time.perf_counter()
    prox(x, 1.0)
    t_prox = time.perf_counter() - t0
    t1 = sum(oracle_gridding_sample(w, x, maps[:1], traj, m1))
    t2 = sum(oracle_gridding_sample(w, x, maps[:2], traj, m1)) if maps.shape[0] > 1 else 2 * t1
    per_coil = max(t2 - t1 - 2 * t_fft, 0.0) / m1                # forward + adjoint, per sample and coil
    per_call = max(t1 - 2 * t_fft - per_coil * m1, 0.0) / m1     # tap tables, per sample
    return {"t_fft_grid": t_fft, "t_prox": t_prox, "G": grid_points(w), "m1": m1, "t1": t1, "t2": t2,
            "grid_per_coil": per_coil, "grid_per_call": per_call}


def oracle_gridding_sample(w, x, maps, traj, m1):
    """The oracle's forward and adjoint NUFFT with the given coils on the first m1 samples (each
    call does one FFT per coil of the oversampled grid and the Kaiser-Bessel gridding)."""
    from oracle import nufft as onf
    sub = traj[:m1]
    t0 = time.perf_counter()
    y1 = onf.nufft_forward(x, maps, sub, w.oversamp, w.width)
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    onf.nufft_adjoint(y1, maps, sub, w.oversamp, w.width)
    t_adj = time.perf_counter() - t0
    return t_fwd, t_adj


def oracle_estimate(w, cal, t1=None):
    """Whole reconstruction time (s) of the float64 oracle, extrapolated from the measured pieces
    (t1: a fresh one-coil forward + adjoint sample time, scaling the calibrated gridding costs).
    Model: one application of A and A^H with C coils costs 2 C grid FFTs + (per-call + C x
    per-coil gridding) x M; the preconditioner (Sec. 5.1 route as the oracle runs it) costs
    C^2 + C FFTs of the 2N image, 1 + C FFTs of its oversampled grid and 1 + C one-coil gridding
    passes; FFT times scale as n log n from the measured single-coil grid FFT.  30 power
    iterations and `iters` PDHG iterations each apply A and A^H; PDHG adds the prox."""
    C, M, N, G = w.ncoils, n_samples(w), int(np.prod(w.img_shape)), cal["G"]
    d = len(w.img_shape)
    tf = cal["t_fft_grid"]
    scale = 1.0 if t1 is None else max(t1 - 2 * tf, 1e-9) / max(cal["t1"] - 2 * tf, 1e-9)
    gc, gt = cal["grid_per_coil"] * scale, cal["grid_per_call"] * scale
    T_AAH = 2 * C * tf + (gt + C * gc) * M
    N2, G2 = N * 2 ** d, G * 2 ** d
    T_pre = ((C * C + C) * tf * _nlogn(N2) / _nlogn(G) + (1 + C) * tf * _nlogn(G2) / _nlogn(G)
             + (1 + C) * 0.5 * (gt + gc) * M)
    T_pow = 30 * T_AAH
    T_pdhg = w.iters * (T_AAH + cal["t_prox"])
    return {"est_s": T_pre + T_pow + T_pdhg, "precond_s": T_pre, "power_s": T_pow, "pdhg_s": T_pdhg,
            "per_iter_s": T_AAH + cal["t_prox"]}


def _sample_m1(w, frac):
    return max(1024, n_samples(w) // frac)


def oracle_sample(w, frac=32):
    """One bounded sample of the float64 oracle on the workload (one host core): the calibration
    above on 1/frac of the samples; returns the extrapolated value."""
    x, maps, traj = oracle_inputs(w)
    t0 = time.perf_counter()
    m1 = _sample_m1(w, frac)
    cal = oracle_calibrate(w, x, maps, traj, m1)
    cpu_s = time.perf_counter() - t0
    est = oracle_estimate(w, cal)
    return {"value": w.iters / est["est_s"], "unit": "iters/s", "cores": 1, "kind": "oracle",
            "sample": (f"float64 NumPy oracle, one core, {cpu_s:.1f} s: a one-coil FFT of the {w.name} "
                       f"oversampled grid ({cal['t_fft_grid']:.2f} s), the prox on the full image "
                       f"({cal['t_prox']:.2f} s), forward + adjoint NUFFT on {m1} of {n_samples(w)} samples "
                       f"with one coil ({cal['t1']:.2f} s) and two coils ({cal['t2']:.2f} s); the whole "
                       f"reconstruction extrapolated by an n log n / per-sample cost model to "
                       f"{est['est_s']:.0f} s (preconditioner {est['precond_s']:.0f} s, 30 power its "
                       f"{est['power_s']:.0f} s, {w.iters} PDHG its {est['pdhg_s']:.0f} s)"),
            "extrapolated_whole_reconstruction_s": est["est_s"]}


def _replica(name, frac):
    return oracle_sample(synth.workload(name), frac)


def oracle_all_cores(w, frac=32):
    """The same one-core sample run as concurrent replicas on every host core (spawned
    processes); value = replicas x the slowest replica's extrapolated iterations per second."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    try:
        import psutil
        avail = psutil.virtual_memory().available
    except Exception:
        avail = 64 << 30
    need = 4 * grid_points(w) * 16 + (2 << 30)                # per replica, generous
    P = int(max(1, min(cores, avail // need)))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(P) as pool:
        res = pool.starmap(_replica, [(w.name, frac)] * P)
    wall = time.perf_counter() - t0
    slow = min(r["value"] for r in res)
    return {"value": P * slow, "unit": "iters/s", "cores": P, "kind": "oracle",
            "sample": f"{P} concurrent replicas of the one-core sample (spawned processes, {wall:.1f} s wall); "
                      f"value = {P} x the slowest replica's extrapolated rate"}


def run_reference(args, rank, world):
    """The float64 oracle as it stands, on the host: each step is one bounded sample (one-coil
    forward and adjoint NUFFT on 1/32 of the workload's samples); the whole reconstruction is
    extrapolated from it and from the calibration measured once before the steps."""
    w = synth.workload(args.workload)
    if rank != 0:
        return
    x, maps, traj = oracle_inputs(w)
    m1 = _sample_m1(w, 32)
    cal = oracle_calibrate(w, x, maps, traj, m1)
    for _ in range(args.warmup):
        oracle_gridding_sample(w, x, maps[:1], traj, m1)
    step_ms, vals = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        t1 = sum(oracle_gridding_sample(w, x, maps[:1], traj, m1))
        step_ms.append(1e3 * (time.perf_counter() - t0))
        vals.append(w.iters / oracle_estimate(w, cal, t1)["est_s"])
    v = statistics.median(vals)
    est_s = w.iters / v
    sample = (f"each step: the float64 NumPy oracle's one-coil forward and adjoint NUFFT on {m1} of "
              f"{n_samples(w)} samples (one host core); calibrated once before the steps: a one-coil grid "
              f"FFT ({cal['t_fft_grid']:.2f} s), the prox ({cal['t_prox']:.2f} s) and the same sample with two "
              f"coils; value = {w.iters} iterations / the whole reconstruction extrapolated by an n log n / "
              f"per-sample cost model")
    line = {"impl": "reference", "metric": metric_name(w), "value": v, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(step_ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w),
            "extrapolated_whole_reconstruction_s": est_s,
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": v, "unit": "iters/s", "sample": sample},
            "e2e": {"value": v, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def algorithmic_bytes(w, C, M, N, G, maps_bytes=8):
    """Algorithmic HBM bytes per PDHG iteration of each phase (each array touched once)."""
    c8, m, D = 8, C * M, len(w.img_shape)
    return {
        "fwd_pre": N * 8 + C * N * maps_bytes + C * G * 8,     # x, maps in; whole grid out
        "interp_dual": C * G * 8 + m * (8 + 4 + 8 + 8) + M * D * 4,   # grid, y, p, u in/out, traj
        "spread": m * c8 + M * D * 4 + C * G * 8,              # u, traj in; whole grid out
        "adj_primal": C * N * 8 + C * N * maps_bytes + N * 8 * 3,   # cropped grid, maps, x in/out, z out
        "fft_fwd": 2 * C * G * 8, "fft_inv": 2 * C * G * 8,     # one read + one write pass
        "dwt_fwd": 2 * 2 * N * 8, "dwt_inv": 2 * 2 * N * 8, "soft": 2 * N * 8, "extrap": 4 * N * 8,
    }


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of kernels of the timed
# workload from one ncu capture, keyed by (workload, phase).  An entry is valid only for the
# kernel code it was taken on; drop it when its kernel changes until it is captured again.
NCU_TRAFFIC = {
    # one capture of the full 3D UTE workload (192^3 x 8 coils, 6,144,000 samples; one pass per
    # kernel, so allowed at full size): KPDHG_SPREAD_VARIANT=10 KPDHG_SPREAD_CHUNK=256 ncu --metrics
    # dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none
    # -k "regex:k_spread_own|k_halo_gather" -s 10 -c 4 python bench.py --steps 1 --warmup 1 --no-extras
    # k_spread_own<float2, 4>: 1.282 GB read + 1.440 GB written; k_halo_gather: 1.527 + 0.854 GB
    ("ute3d_192", "spread"): {"bytes": 5103672448,
                              "kernel": "k_spread_own<float2, 4> + k_halo_gather (one launch each, full 3D UTE workload)"},
}

# Relative l2 errors against the float64 oracle measured by the GPU parity tests for the forms
# reported beside the plain solver (the largest value each test logged, KPDHG_PARITY_LOG, on a
# GB300 with the spreading and interpolation kernels of this tree).  "stored inputs": oracle fed
# the same 16-bit values; "storage error": oracle on the unrounded inputs.  The tests hold the
# pass/fail tolerances (1e-5 float32, 2e-3 storage).
ORACLE_ERRORS = {
    "ute3d_192_operators": {"forward": 3.08e-07, "adjoint": 7.44e-07,
                            "test": "test_gpu_nufft.py::test_forward_adjoint_3d_ute_full_size (every sample)"},
    "ute3d_own_fft_passes": {"forward": 6.9e-07, "adjoint": 6.19e-07,
                             "test": "test_gpu_nufft.py::test_own_fft_passes_match_oracle_and_cufft (every compiled length, 20-480)"},
    "ute3d_pdhg_small": {"precond": 5.44e-07, "x": 3.02e-07, "test": "test_gpu_pdhg.py::test_pdhg_3d_parity"},
    "fp16_maps_3d_pdhg": {"stored_inputs": 3.06e-07, "storage_error": 1.2e-04,
                          "test": "test_gpu_pdhg.py::test_pdhg_3d_fp16_maps (16^3 x 3 coils, 20 l1 iterations)"},
    "spiral2d_256_pdhg_100": {"x": 3.66e-07, "test": "test_gpu_pdhg.py::test_pdhg_full_chain_workloads (GPU p and L)"},
    "bf16_kspace_fp16_maps_pdhg": {"stored_inputs": 3.01e-07, "storage_error": 3.92e-04,
                                   "test": "test_gpu_pdhg.py::test_pdhg_half_storage[bf16-fp16] (64^2 x 4, 30 l1 its)"},
    "batched_bf16_kspace": {"stored_inputs": 6.96e-07, "storage_error": 1.23e-03,
                            "test": "test_gpu_batch.py::test_batch_uneven_bf16_kspace_against_oracle (3 uneven cases)"},
    "batched_c64": {"x": 1.42e-06, "test": "test_gpu_batch.py::test_batch_matches_oracle_and_single_solves"},
    "batched_phase_form": {"x": 1.39e-06, "test": "test_gpu_batch.py::test_batch_phase_form"},
    "host_measurements": {"x_vs_device_y": 5.08e-07,
                          "test": "test_gpu_state_and_failures.py::test_host_measurements_overlap_the_setup"},
    "unrolled_grad": {"x": 2.64e-07, "dL_dy": 1.42e-06, "dL_dtraj": 1.05e-06,
                      "test": "test_gpu_autograd.py::test_unrolled_gradients_match_oracle"},
}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "MEASURED_PEAKS.json hbm_gbs"
    except Exception:
        return {}, "fallback 6800 GB/s"


class Recon:
    """One workload's plan, device inputs and pinned host copies (synthetic measurements
    y = A x + 1 % complex Gaussian noise made by the GPU's own forward operator)."""

    def __init__(self, w, dev, maps_storage=None, y_storage=None):
        import torch
        from paper_1902_09657_gb300.api import Plan, to_storage
        self.w, self.dev = w, dev
        ms, ys = storage_of(w)
        self.maps_storage = maps_storage or ms
        self.y_storage = y_storage or ys
        self.traj_h = torch.from_numpy(w.traj()).pin_memory()
        self.C, self.M = w.ncoils, self.traj_h.shape[0]
        self.N, self.G = int(np.prod(w.img_shape)), grid_points(w)
        self.traj_d = self.traj_h.to(dev)
        maps = torch.from_numpy(w.maps()).to(dev)
        self.maps_d = to_storage(maps, self.maps_storage)
        self.maps_h = self.maps_d.cpu().pin_memory()
        self.plan = Plan(w.img_shape, self.C, self.M, oversamp=w.oversamp, wavelet_levels=w.wavelet_levels,
                         device=dev)
        self.plan.set_trajectory(self.traj_d).set_maps(self.maps_d)
        y = self.plan.sense_forward(torch.from_numpy(w.phantom()).to(dev))
        noise = torch.from_numpy(w.noise().astype(np.complex64)).to(dev)
        y = (y + 0.01 * y.abs().max() * noise).contiguous()
        self.lam = lambda_for(w, ahy_max=float(self.plan.sense_adjoint(y).abs().max()))
        self.y_d = to_storage(y, self.y_storage)
        self.y_h = self.y_d.cpu().pin_memory()

    def step(self):
        self.plan.set_trajectory(self.traj_d).set_maps(self.maps_d)
        return self.plan.pdhg_solve(self.y_d, None, self.w.reg, self.lam, self.w.iters)

    def close(self):
        self.plan.close()


def _timed(fn, stream, flush, reps):
    """Mean device time (ms) of fn() over reps runs, L2 flushed before each."""
    import torch
    tot = 0.0
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / reps


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1902_09657_gb300 import _build

    _build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = synth.workload(args.workload)
    rc = Recon(w, dev)
    plan = rc.plan
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        rc.step()
    torch.cuda.synchronize()
    launches0 = plan.launch_count()
    clocks = Clocks(dev.index if "CUDA_VISIBLE_DEVICES" not in os.environ else local_rank)
    clocks.start()
    total_ms = 0.0
    barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc.step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    launches = plan.launch_count() - launches0
    total_ms = max_over_ranks(total_ms, world, dev)
    value = whole_job_value(world, args.steps, w.iters, total_ms)

    extras = {}
    if not args.no_extras and rank == 0:
        extras = gpu_extras(rc, stream, flush, args, world)
    if rank != 0:
        return
    line = {"metric": metric_name(w), "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(w), "clocks": ck, "gpu_launches": int(launches)}
    line.update(extras)
    print(json.dumps(line), flush=True)


def e2e_through_api(rc, stream, flush, k):
    """The whole reconstruction through the public API with host buffers: pinned traj, maps and
    y copied in (y by the library, overlapping the set-up) and x copied back into a pinned
    buffer inside each timed step."""
    import torch
    w, plan, dev = rc.w, rc.plan, rc.dev
    x_h = torch.empty(w.img_shape, dtype=torch.complex64).pin_memory()     # the caller's result buffer
    tot = 0.0
    for i in range(k + 1):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        td = rc.traj_h.to(dev, non_blocking=True)
        md = rc.maps_h.to(dev, non_blocking=True)
        plan.set_trajectory(td).set_maps(md)
        plan.pdhg_solve(rc.y_h, None, w.reg, rc.lam, w.iters, out=x_h)
        e1.record(stream)
        e1.synchronize()
        if i > 0:
            tot += e0.elapsed_time(e1)
    el = lambda t: t.numel() * t.element_size()
    return {"value": k * w.iters / (tot / 1e3), "unit": "iters/s",
            "h2d_bytes_per_step": int(el(rc.traj_h) + el(rc.maps_h) + el(rc.y_h)),
            "d2h_bytes_per_step": int(rc.N * 8)}


def setup_and_solve(rc, stream):
    """Set-up (binning, maps, MC preconditioner, 30 power iterations) and solve-only times."""
    import torch
    w, plan = rc.w, rc.plan
    ev = lambda: torch.cuda.Event(enable_timing=True)
    plan.set_trajectory(rc.traj_d).set_maps(rc.maps_d)
    torch.cuda.synchronize()
    e0, ea, eb, e1, e2 = ev(), ev(), ev(), ev(), ev()
    e0.record(stream)
    plan.set_trajectory(rc.traj_d).set_maps(rc.maps_d)
    ea.record(stream)
    p = plan.make_preconditioner(True)
    eb.record(stream)
    L = plan.max_eig(p, iters=30)
    e1.record(stream)
    plan.pdhg_solve(rc.y_d, p, w.reg, rc.lam, w.iters, lmax=L)
    e2.record(stream)
    e2.synchronize()
    rc.setup_parts = {"trajectory_and_maps_ms": e0.elapsed_time(ea), "preconditioner_ms": ea.elapsed_time(eb),
                      "power_method_ms": eb.elapsed_time(e1)}
    return p, L, e0.elapsed_time(e1), e1.elapsed_time(e2)


def phase_profile(rc, p, L, k):
    """Per-phase GPU time per iteration (events at every phase boundary, no graph)."""
    plan, w = rc.plan, rc.w
    plan.set_profiling(True)
    _, _, st = plan.pdhg_solve(rc.y_d, p, w.reg, rc.lam, k, lmax=L)
    plan.set_profiling(False)
    return {n: v / k for n, v in st["phase_ms"].items() if v > 0}


def roofline(rc, ph):
    """Dominant own phase of the profiled iteration: algorithmic bytes / its mean duration
    against the measured HBM copy bandwidth."""
    w = rc.w
    mb = 4 if rc.maps_storage != "c64" else 8
    ab = algorithmic_bytes(w, rc.C, rc.M, rc.N, rc.G, maps_bytes=mb)
    own = {n: v for n, v in ph.items() if n in ab and not n.startswith("fft")}
    if "spread" in own and "spread_reduce" in ph:          # two-phase spreading: both kernels
        own["spread"] += ph["spread_reduce"]
    dom = max(own, key=own.get)
    peaks, psrc = _peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = ab[dom] / (own[dom] * 1e-3) / 1e9
    tr = NCU_TRAFFIC.get((w.name, dom))
    kern = {"spread": "spreading (k_spread_own + k_halo_gather)" if "spread_reduce" in ph else "spreading",
            "interp_dual": "k_interp_tile (interpolation + dual step)",
            "adj_primal": "primal step (k_primal_fused / k_adj_primal)"}.get(dom, dom)
    out = {"kernel": kern, "phase": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "traffic": tr["bytes"] if tr else None,
           "traffic_source": ("one ncu capture of " + tr["kernel"]) if tr else None,
           "peak_source": psrc, "algorithmic_bytes": int(ab[dom]), "avg_launch_ms": own[dom]}
    per = {}
    for n, v in ph.items():
        b = ab.get(n)
        if n == "spread" and "spread_reduce" in ph:
            v = v + ph["spread_reduce"]
        per[n] = {"ms": round(v, 5)}
        if b:
            per[n].update(GB_per_s=round(b / (v * 1e-3) / 1e9, 1), frac=round(b / (v * 1e-3) / 1e9 / peak, 4))
    return out, per


def time_to_accuracy(rc, p, L, setup_ms, solve_ms, long_iters):
    """Iterations and time until (F(x_k) - F*)/|F*| < 1e-3, F* the least objective of a
    long_iters float32 GPU run from the same start (1000 iterations for 3D)."""
    w, plan = rc.w, rc.plan
    _, tr, _ = plan.pdhg_solve(rc.y_d, p, w.reg, rc.lam, long_iters, lmax=L, trace=True)
    Fstar = min(tr)
    kk = next((i + 1 for i, f in enumerate(tr) if (f - Fstar) / abs(Fstar) < 1e-3), None)
    per_it = solve_ms / w.iters
    return {"iters": kk, "ms_solve_only": None if kk is None else kk * per_it,
            "ms_with_setup": None if kk is None else setup_ms + kk * per_it,
            "F_star": Fstar, "F_star_source": f"min of a {long_iters}-iteration float32 GPU run"}


def nufft_rates(rc, stream, flush):
    """Forward (type-2) and adjoint (type-1) SENSE NUFFT: coil-sample points per second."""
    import torch
    plan = rc.plan
    x = plan.sense_adjoint(rc.y_d)
    yo = torch.empty((rc.C, rc.M), dtype=torch.complex64, device=rc.dev)
    for _ in range(2):
        plan.sense_forward(x, out=yo)
        plan.sense_adjoint(yo, out=x)
    t_f = _timed(lambda: plan.sense_forward(x, out=yo), stream, flush, 5)
    t_a = _timed(lambda: plan.sense_adjoint(yo, out=x), stream, flush, 5)
    cm = rc.C * rc.M
    return {"forward_ms": t_f, "adjoint_ms": t_a, "forward_Mpts_per_s": cm / (t_f * 1e3),
            "adjoint_Mpts_per_s": cm / (t_a * 1e3)}


def gpu_extras(rc, stream, flush, args, world):
    import torch
    w = rc.w
    out = {}
    out["e2e"] = e2e_through_api(rc, stream, flush, max(1, min(args.steps, 5)))
    p, L, setup_ms, solve_ms = setup_and_solve(rc, stream)
    out["setup_ms"] = setup_ms
    out["setup_parts"] = rc.setup_parts
    out["solve_only_iters_per_s"] = w.iters / (solve_ms / 1e3)
    ph = phase_profile(rc, p, L, 5 if w.name == "ute3d_192" else w.iters)
    out["roofline"], out["phase_per_iter"] = roofline(rc, ph)
    out["spread_config"] = rc.plan.spread_config()
    out["nufft"] = nufft_rates(rc, stream, flush)
    out["time_to_1e-3"] = time_to_accuracy(rc, p, L, setup_ms, solve_ms, 1000 if len(w.img_shape) == 3 else 400)
    if not args.no_side_workloads:
        rc.close()
        torch.cuda.empty_cache()
        for key, fn in (("spiral2d_256", side_spiral), ("radial2d_128", side_radial),
                        ("batched_64", side_batched), ("unrolled_grad", side_unrolled)):
            try:
                out[key] = fn(rc.dev, stream, flush)
            except Exception as e:  # reported, never hidden
                out[key] = {"error": repr(e)}
            torch.cuda.empty_cache()
    if ORACLE_ERRORS:
        out["oracle_errors"] = ORACLE_ERRORS
    if world == 1:
        try:
            out["cpu_baseline"] = oracle_sample(w)
            out["cpu_baseline_all_cores"] = oracle_all_cores(w)
        except Exception as e:  # reported, never hidden
            out["cpu_baseline"] = {"error": repr(e)}
    return out


def whole_reconstruction(name, dev, stream, flush, reps=5, maps_storage=None, y_storage=None):
    """Whole reconstructions of a workload per second (as the headline step), set-up and solve."""
    w = synth.workload(name)
    rc = Recon(w, dev, maps_storage, y_storage)
    for _ in range(2):
        rc.step()
    t = _timed(rc.step, stream, flush, reps)
    p, L, setup_ms, solve_ms = setup_and_solve(rc, stream)
    res = {"iters_per_s": w.iters / (t / 1e3), "ms_per_reconstruction": t, "setup_ms": setup_ms,
           "solve_only_iters_per_s": w.iters / (solve_ms / 1e3), "maps": rc.maps_storage, "y": rc.y_storage}
    return rc, p, L, setup_ms, solve_ms, res


def side_spiral(dev, stream, flush):
    """2D spiral l1-wavelet (256^2 x 12 coils, 24 x 4096, 100 iterations): whole reconstruction,
    the per-phase profile, time to 1e-3, the convergence of Sec. 6's comparison (no / single- /
    multi-channel preconditioner), TV (Sec. 4.2), and the BF16-k-space / FP16-maps variant."""
    import torch
    rc, p, L, setup_ms, solve_ms, res = whole_reconstruction("spiral2d_256", dev, stream, flush)
    w, plan = rc.w, rc.plan
    ph = phase_profile(rc, p, L, w.iters)
    res["roofline"], res["phase_per_iter"] = roofline(rc, ph)
    res["spread_config"] = plan.spread_config()
    res["time_to_1e-3"] = time_to_accuracy(rc, p, L, setup_ms, solve_ms, 400)
    res["comparison_sec6"] = method_comparison(rc, stream, flush, 300)
    plan.pdhg_solve(rc.y_d, p, "tv", rc.lam, w.iters, lmax=L)
    tv_ms = _timed(lambda: plan.pdhg_solve(rc.y_d, p, "tv", rc.lam, w.iters, lmax=L), stream, flush, 3)
    res["tv_solve_only"] = {"iters": w.iters, "ms": tv_ms, "iters_per_s": w.iters / (tv_ms * 1e-3),
                            "steps": "sigma = theta = 1, tau = 1/(L + 4 ndim)"}
    x32, _, _ = plan.pdhg_solve(rc.y_d, p, w.reg, rc.lam, w.iters, lmax=L)
    rc.close()
    rh, _, _, _, _, half = whole_reconstruction("spiral2d_256", dev, stream, flush, 5, "fp16", "bf16")
    xh, _, _ = rh.plan.pdhg_solve(rh.y_d, p, w.reg, rh.lam, w.iters, lmax=L)
    half["rel_diff_vs_fp32_storage"] = float((xh - x32).norm() / x32.norm())
    rh.close()
    res["bf16_kspace_fp16_maps"] = half
    return res


def side_radial(dev, stream, flush):
    """2D golden-angle radial l2 (128^2 x 4 coils, 64 x 256, alpha 2, 30 iterations), with the
    comparison of Sec. 6 (CG, circulant-preconditioned CG, FISTA, PDHG without preconditioner,
    single- and multi-channel)."""
    rc, p, L, setup_ms, solve_ms, res = whole_reconstruction("radial2d_128", dev, stream, flush, reps=10)
    res["time_to_1e-3"] = time_to_accuracy(rc, p, L, setup_ms, solve_ms, 400)
    res["comparison_sec6"] = method_comparison(rc, stream, flush, 300)
    rc.close()
    return res


def method_comparison(rc, stream, flush, iters):
    """Sec. 6's comparison on one workload: objective traces of `iters` iterations of every
    method, F* the least objective any reaches; per method the iterations and the time to a
    relative objective (F - F*)/|F*| of 1e-2 and 1e-3, and the time per iteration (untraced
    solves, L2 flushed).  Set-up (preconditioners, power method) is timed separately."""
    import torch
    w, plan, dev = rc.w, rc.plan, rc.dev
    y, lam, reg = rc.y_d, rc.lam, w.reg
    runs = {}
    for name in ("none", "single_channel", "multi_channel"):
        pp = torch.ones((rc.C, rc.M), dtype=torch.float32, device=dev) if name == "none" else \
            plan.make_preconditioner(name == "multi_channel")
        Lp = plan.max_eig(pp, iters=30)
        _, trc, _ = plan.pdhg_solve(y, pp, reg, lam, iters, lmax=Lp, trace=True)
        t = _timed(lambda: plan.pdhg_solve(y, pp, reg, lam, 50, lmax=Lp), stream, flush, 3) / 50
        runs["pdhg_" + name] = (list(trc), t, {"lmax": Lp})
    if reg == "l2":
        for name, circ in (("cg", False), ("cg_circulant", True)):
            plan.circulant_preconditioner()
            _, trc = plan.cg_l2_solve(y, lam, iters, circulant=circ)
            t = _timed(lambda: plan.cg_l2_solve(y, lam, 50, circulant=circ, trace=False), stream, flush, 3) / 50
            runs[name] = (list(trc), t, {})
    La = 1.01 * plan.max_eig(None, iters=30)
    _, trc = plan.fista_solve(y, reg, lam, iters, lmax=La)
    t = _timed(lambda: plan.fista_solve(y, reg, lam, 50, lmax=La, trace=False), stream, flush, 3) / 50
    runs["fista"] = (list(trc), t, {"L": La})
    Fs = min(min(tr) for tr, _, _ in runs.values())
    out = {"F_star": Fs, "F_star_source": f"least objective of {iters} iterations of every method (float32 GPU)",
           "iters": iters}
    for name, (trc, t, extra) in runs.items():
        rel_obj = [(f - Fs) / abs(Fs) for f in trc]
        k2 = next((i + 1 for i, r in enumerate(rel_obj) if r < 1e-2), None)
        k3 = next((i + 1 for i, r in enumerate(rel_obj) if r < 1e-3), None)
        out[name] = dict(extra, ms_per_iter=t, iters_to_1e_2=k2, iters_to_1e_3=k3,
                         ms_to_1e_3=None if k3 is None else k3 * t, rel_obj_at_30=rel_obj[min(29, len(rel_obj) - 1)])
    return out


def _measure_y(plan, x, gen):
    import torch
    y = plan.sense_forward(x)
    n = torch.randn(y.shape, dtype=torch.complex64, device=y.device, generator=gen)
    return (y + 0.01 * y.abs().max() * n).contiguous()


def side_batched(dev, stream, flush, n_cases=64, iters=20):
    """64 uneven cases (96..320 image, 4..32 coils, radial/spiral, l2/l1) with BF16 k-space:
    one kp_batch solve (per-case MC preconditioner + 30 power iterations, then `iters`
    graph-replayed iterations of all cases at once) against the same cases solved one after
    another."""
    import torch
    from paper_1902_09657_gb300.api import Batch, Plan, to_storage
    gen = torch.Generator(device=dev).manual_seed(11)
    cases = synth.batched_cases(n_cases)
    plans, ys, lams, regs = [], [], [], []
    samples = 0
    for w in cases:
        traj = torch.from_numpy(w.traj()).to(dev)
        plan = Plan(w.img_shape, w.ncoils, traj.shape[0], oversamp=w.oversamp, wavelet_levels=w.wavelet_levels,
                    device=dev)
        plan.set_trajectory(traj).set_maps(torch.from_numpy(w.maps()).to(dev))
        y = _measure_y(plan, torch.from_numpy(w.phantom()).to(dev), gen)
        lam = w.lam_rel * (float(plan.sense_adjoint(y).abs().max()) if w.reg == "l1_wavelet" else 1.0)
        plans.append(plan)
        ys.append(to_storage(y, "bf16"))
        lams.append(lam)
        regs.append(w.reg)
        samples += w.ncoils * traj.shape[0]
    batch = Batch(plans)
    batch.solve(ys, None, regs, lams, iters)          # captures the all-case graph
    t_batch = _timed(lambda: batch.solve(ys, None, regs, lams, iters), stream, flush, 3)
    t_setup = _timed(lambda: batch.solve(ys, None, regs, lams, 0), stream, flush, 3)
    batch.set_form("phases")
    batch.solve(ys, None, regs, lams, iters)
    t_phases = _timed(lambda: batch.solve(ys, None, regs, lams, iters), stream, flush, 3)
    batch.set_form("per_case")

    def sequential():
        for pl, y, r, lm in zip(plans, ys, regs, lams):
            pl.pdhg_solve(y, None, r, lm, iters)
    sequential()
    t_seq = _timed(sequential, stream, flush, 3)
    batch.close()
    for pl in plans:
        pl.close()
    return {"cases": n_cases, "iters": iters, "coil_samples": int(samples), "y": "bf16",
            "batched_ms": t_batch, "batched_cases_per_s": n_cases / (t_batch / 1e3),
            "batched_setup_ms": t_setup, "batched_iteration_ms": (t_batch - t_setup) / iters,
            "phase_form_ms": t_phases, "phase_form_iteration_ms": (t_phases - t_setup) / iters,
            "sequential_ms": t_seq, "sequential_cases_per_s": n_cases / (t_seq / 1e3),
            "what": "whole reconstructions (MC preconditioner, 30 power its, PDHG its) per second"}


def side_unrolled(dev, stream, flush):
    """Differentiable unrolled l2 PDHG (256^2 spiral, 16 coils, 16 x 4096, 10 iterations):
    forward with per-iteration checkpoints, and the reverse sweep giving dL/dy, dL/dlambda and
    the trajectory gradient."""
    import torch
    from paper_1902_09657_gb300.api import Plan
    w = synth.workload("spiral2d_256_unrolled")
    traj = torch.from_numpy(w.traj()).to(dev)
    M, C = traj.shape[0], w.ncoils
    plan = Plan(w.img_shape, C, M, oversamp=w.oversamp, device=dev)
    plan.set_trajectory(traj).set_maps(torch.from_numpy(w.maps()).to(dev))
    gen = torch.Generator(device=dev).manual_seed(5)
    y = _measure_y(plan, torch.from_numpy(w.phantom()).to(dev), gen)
    p = plan.make_preconditioner(True)
    L = plan.max_eig(p, iters=30)
    gx = torch.randn(w.img_shape, dtype=torch.complex64, device=dev, generator=gen)
    for _ in range(3):
        plan.unrolled_forward(y, p, w.lam_rel, w.iters, L)
        plan.unrolled_backward(gx)
    t_f = _timed(lambda: plan.unrolled_forward(y, p, w.lam_rel, w.iters, L), stream, flush, 5)
    t_b = _timed(lambda: plan.unrolled_backward(gx), stream, flush, 5)
    plan.close()
    return {"iters": w.iters, "forward_ms": t_f, "backward_ms": t_b,
            "backward_outputs": "dL/dy, dL/dlambda, dL/dtraj"}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
