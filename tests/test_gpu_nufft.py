"""GPU parity of the SENSE NUFFT pair (Sec. 2 Eq. model_i; Sec. 6 KB gridding) against the
float64 oracle, through the C ABI.  Tolerance: relative l2 1e-5 for float32 operators, and
the storage rounding bound for half storage (bf16 2^-9, fp16 2^-12 per element)."""
import numpy as np
import pytest

from oracle import nufft as onf
from tests.gpu_util import need_gpu, rel, random_problem, workload_problem, to_dev, make_plan, torch

pytestmark = pytest.mark.gpu

CASES = [
    # (shape, coils, samples, oversampling, seed): ragged grids spanning several tiles
    ((40, 56), 3, 1500, 1.25, 1),
    ((64, 64), 1, 1, 1.25, 2),
    ((8, 8), 2, 37, 2.0, 3),
    ((16, 20, 12), 2, 900, 1.25, 4),
    ((24, 24, 24), 3, 2000, 1.25, 5),
]


@pytest.mark.parametrize("shape,C,M,alpha,seed", CASES)
def test_forward_adjoint_random(shape, C, M, alpha, seed):
    need_gpu()
    x, maps, traj = random_problem(shape, C, M, seed, edge=True)
    y_ref = onf.nufft_forward(x.astype(np.complex128), maps.astype(np.complex128), traj, alpha, 4)
    u = (np.random.default_rng(seed + 100).standard_normal((C, M))
         + 1j * np.random.default_rng(seed + 101).standard_normal((C, M))).astype(np.complex64)
    x_ref = onf.nufft_adjoint(u.astype(np.complex128), maps.astype(np.complex128), traj, alpha, 4)
    plan = make_plan(shape, C, M, alpha)
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    y = plan.sense_forward(to_dev(x)).cpu().numpy()
    xa = plan.sense_adjoint(to_dev(u)).cpu().numpy()
    assert rel(y, y_ref) < 1e-5
    assert rel(xa, x_ref) < 1e-5
    # adjoint identity of the GPU pair itself
    lhs = np.vdot(u.astype(np.complex128), y.astype(np.complex128))
    rhs = np.vdot(xa.astype(np.complex128), x.astype(np.complex128))
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)


@pytest.mark.parametrize("name,alpha", [("radial2d_128", 2.0), ("spiral2d_256", 1.25)])
def test_forward_adjoint_workloads(name, alpha):
    """Full-size 2D workloads (golden-angle radial 128^2 x 4 coils; spiral 256^2 x 12 coils)."""
    need_gpu()
    w, x, maps, traj = workload_problem(name)
    C, M = maps.shape[0], traj.shape[0]
    y_ref = onf.nufft_forward(x.astype(np.complex128), maps.astype(np.complex128), traj, alpha, 4)
    x_ref = onf.nufft_adjoint(y_ref, maps.astype(np.complex128), traj, alpha, 4)
    plan = make_plan(x.shape, C, M, alpha)
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    y = plan.sense_forward(to_dev(x)).cpu().numpy()
    xa = plan.sense_adjoint(to_dev(y_ref.astype(np.complex64))).cpu().numpy()
    assert rel(y, y_ref) < 1e-5
    assert rel(xa, x_ref) < 1e-5
    nt, mx = plan.tile_stats()
    assert nt > 0 and mx > 0


def test_forward_adjoint_3d_ute_full_size():
    """3D centre-out radial 192^3 x 8 coils x 6,144,000 samples (the 3D workload) in the launch
    configuration the solver uses (autotuned spreading, two-phase for this trajectory): forward
    and adjoint on every sample and pixel against the float64 oracle (a 240^3 x 8 float64 grid
    on the host)."""
    need_gpu()
    w, x, maps, traj = workload_problem("ute3d_192")
    C, M = maps.shape[0], traj.shape[0]
    plan = make_plan(x.shape, C, M, 1.25)
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    cfg = plan.spread_config()
    y = plan.sense_forward(to_dev(x)).cpu().numpy()
    rng = np.random.default_rng(17)
    u = (rng.standard_normal((C, M), dtype=np.float32) + 1j * rng.standard_normal((C, M), dtype=np.float32))
    xa = plan.sense_adjoint(to_dev(u.astype(np.complex64))).cpu().numpy()
    plan.close()
    m128 = maps.astype(np.complex128)
    y_ref = onf.nufft_forward(x.astype(np.complex128), m128, traj, 1.25, 4)
    assert rel(y, y_ref, "forward") < 1e-5
    del y_ref
    x_ref = onf.nufft_adjoint(u, m128, traj, 1.25, 4)
    assert rel(xa, x_ref, f"adjoint, spreading variant {cfg['variant']}") < 1e-5, cfg


@pytest.mark.parametrize("ystore,mstore", [("bf16", "c64"), ("fp16", "c64"), ("c64", "fp16"), ("c64", "bf16"),
                                           ("bf16", "fp16"), ("fp16", "fp16"), ("bf16", "bf16")])
def test_half_storage(ystore, mstore):
    """16-bit storage with float32 arithmetic.  Arithmetic parity: on the stored (rounded) maps
    and data the GPU gives the oracle's result on those same values to 1e-5 (the forward output
    itself is then rounded once more when it is stored in 16 bits).  Storage error: against the
    oracle on the unrounded inputs the result is within 2e-3 whenever at most one bf16 rounding
    is involved; bf16 keeps 8 significant bits, 1.7e-3 relative per rounding, so bf16 maps
    with bf16 data (2.3e-3) are held to arithmetic parity only."""
    need_gpu()
    from paper_1902_09657_gb300.api import to_storage
    from tests.gpu_util import rounded
    shape, C, M = (48, 40), 4, 3000
    x, maps, traj = random_problem(shape, C, M, 7)
    md = to_storage(to_dev(maps), mstore)
    m_r = rounded(md).reshape(maps.shape)
    two_bf16 = ystore == "bf16" and mstore == "bf16"
    plan = make_plan(shape, C, M)
    plan.set_trajectory(to_dev(traj)).set_maps(md)
    # forward with the stored maps; output stored in ystore
    y = plan.sense_forward(to_dev(x), storage=ystore)
    yg = rounded(y).reshape(C, M)
    y_rm = onf.nufft_forward(x.astype(np.complex128), m_r, traj, 1.25, 4)
    y_unr = onf.nufft_forward(x.astype(np.complex128), maps.astype(np.complex128), traj, 1.25, 4)
    out_round = {"c64": 1e-5, "fp16": 4e-4, "bf16": 2e-3}[ystore]
    assert rel(yg, y_rm, "forward, stored maps") < out_round
    e = rel(yg, y_unr, "forward storage error")
    if not two_bf16:
        assert e < 2e-3
    # adjoint of data stored in ystore with the stored maps
    yd = to_storage(to_dev(y_unr.astype(np.complex64)), ystore)
    xa = plan.sense_adjoint(yd).cpu().numpy()
    x_rr = onf.nufft_adjoint(rounded(yd).reshape(C, M), m_r, traj, 1.25, 4)
    assert rel(xa, x_rr, "adjoint, stored inputs") < 1e-5
    x_unr = onf.nufft_adjoint(y_unr, maps.astype(np.complex128), traj, 1.25, 4)
    e = rel(xa, x_unr, "adjoint storage error")
    if not two_bf16:
        assert e < 2e-3


def test_invalid_trajectory_rejected():
    need_gpu()
    from paper_1902_09657_gb300._lib import KpError, KP_EINVAL
    x, maps, traj = random_problem((32, 32), 2, 100, 9)
    traj[5, 0] = 16.5
    plan = make_plan((32, 32), 2, 100)
    with pytest.raises(KpError) as ei:
        plan.set_trajectory(to_dev(traj))
    assert ei.value.status == KP_EINVAL
    traj[5, 0] = np.nan
    with pytest.raises(KpError):
        plan.set_trajectory(to_dev(traj))


def test_invalid_params_rejected():
    need_gpu()
    from paper_1902_09657_gb300._lib import KpError
    from paper_1902_09657_gb300.api import Plan
    with pytest.raises(KpError):
        Plan((32, 32), 2, 100, kernel_width=6)
    with pytest.raises(KpError):
        Plan((30, 32), 2, 100, wavelet_levels=3)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12])
@pytest.mark.parametrize("chunk", [256, 1024])
def test_spread_variants_and_item_sizes(variant, chunk, monkeypatch):
    """Every spreading kernel variant and work-item size (fixed through the tuning overrides)
    gives the oracle's adjoint, on centre-dense radial trajectories whose central tiles are
    cut into many items (2D and 3D; variants 8 to 11 exist in 3D only, 12 in 2D only).  The 3D case has 2
    coils, so coil groups are partly empty."""
    need_gpu()
    import synth
    monkeypatch.setenv("KPDHG_SPREAD_VARIANT", str(variant))
    monkeypatch.setenv("KPDHG_SPREAD_CHUNK", str(chunk))
    cases = [((48, 48), 3, synth.radial_golden_angle(n_spokes=150, n_readout=96, kmax=24.0)),
             ((16, 16, 16), 2, synth.radial_3d_fibonacci(n_spokes=600, n_readout=16, kmax=8.0)),
             ((12, 12, 12), 10, synth.radial_3d_fibonacci(n_spokes=300, n_readout=12, kmax=6.0))]
    for shape, C, traj in cases:
        if (8 <= variant <= 11 and len(shape) == 2) or (variant == 12 and len(shape) == 3):
            continue                                  # variants 8-11 are 3D kernels, 12 is 2D
        M = traj.shape[0]
        rng = np.random.default_rng(M)
        maps = (rng.standard_normal((C,) + shape) + 1j * rng.standard_normal((C,) + shape)).astype(np.complex64)
        u = (rng.standard_normal((C, M)) + 1j * rng.standard_normal((C, M))).astype(np.complex64)
        x_ref = onf.nufft_adjoint(u.astype(np.complex128), maps.astype(np.complex128), traj, 1.25, 4)
        plan = make_plan(shape, C, M, 1.25)
        plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
        cfg = plan.spread_config()
        assert cfg["variant"] == variant and cfg["chunk"] == chunk
        assert cfg["split_tiles"] > 0 or variant >= 10
        xa = plan.sense_adjoint(to_dev(u)).cpu().numpy()
        assert rel(xa, x_ref) < 1e-5, (shape, cfg)


# Image sizes whose 1.25x grids (rounded up to even) have the prime factors 2, 3, 5, 7 and 13
# on either axis, with ragged tiles.
GRID_CASES = [
    (32, 32),       # 40 x 40
    (48, 40),       # 60 x 50
    (56, 44),       # 70 x 56
    (100, 40),      # 126 x 50
    (20, 100),      # 26 x 126
]


@pytest.mark.parametrize("shape", GRID_CASES)
def test_forward_adjoint_grid_sizes(shape):
    """Forward and adjoint against the oracle on grids of mixed-radix and prime-factor sizes."""
    need_gpu()
    C, M = 3, 2500
    x, maps, traj = random_problem(shape, C, M, 11, edge=True)
    u = (np.random.default_rng(12).standard_normal((C, M))
         + 1j * np.random.default_rng(13).standard_normal((C, M))).astype(np.complex64)
    y_ref = onf.nufft_forward(x.astype(np.complex128), maps.astype(np.complex128), traj, 1.25, 4)
    x_ref = onf.nufft_adjoint(u.astype(np.complex128), maps.astype(np.complex128), traj, 1.25, 4)
    plan = make_plan(shape, C, M, 1.25)
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    assert rel(plan.sense_forward(to_dev(x)).cpu().numpy(), y_ref) < 1e-5
    assert rel(plan.sense_adjoint(to_dev(u)).cpu().numpy(), x_ref) < 1e-5


# 3D grids whose sizes factor into 2, 3 and 5 use the library's own FFT passes (pruned to the
# image band); others fall back to cuFFT.  (15, 16, 24) -> grid (20, 20, 30): an odd image edge
# and radix-5 and radix-3 stages; (20, 21, 32) -> grid (26, 28, 40): 26 = 2 x 13 is not
# handled, so that plan runs cuFFT.  The other shapes give every compiled pass length: (48, 64,
# 80) -> 60, 80, 100; (96, 128, 160) -> 120, 160, 200; (192, 256, 307) -> 240, 320, 384 (the
# 192^3 workload's grid edge and its preconditioner's); (320, 16, 384) -> 400, 20, 480.
@pytest.mark.parametrize("shape,C,M,seed", [((15, 16, 24), 3, 2500, 41), ((32, 32, 32), 2, 4000, 42),
                                            ((20, 21, 32), 2, 1500, 43), ((48, 64, 80), 2, 3000, 44),
                                            ((96, 128, 160), 2, 3000, 45), ((192, 256, 307), 1, 2000, 46),
                                            ((320, 16, 384), 2, 2000, 47)])
def test_own_fft_passes_match_oracle_and_cufft(shape, C, M, seed, monkeypatch):
    need_gpu()
    x, maps, traj = random_problem(shape, C, M, seed, edge=True)
    monkeypatch.setenv("KPDHG_FFT", "own")
    plan = make_plan(shape, C, M)
    monkeypatch.setenv("KPDHG_FFT", "cufft")
    ref_plan = make_plan(shape, C, M)
    monkeypatch.delenv("KPDHG_FFT")
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    ref_plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    y = plan.sense_forward(to_dev(x)).cpu().numpy()
    y_cu = ref_plan.sense_forward(to_dev(x)).cpu().numpy()
    y_o = onf.nufft_forward(x.astype(np.complex128), maps.astype(np.complex128), traj, 1.25, 4)
    assert rel(y, y_o, "forward, own FFT passes vs oracle") < 1e-5
    assert rel(y, y_cu, "forward, own FFT passes vs cuFFT") < 2e-6
    yr = (np.random.default_rng(seed).standard_normal(y.shape) + 1j * np.random.default_rng(seed + 1).standard_normal(y.shape)).astype(np.complex64)
    xa = plan.sense_adjoint(to_dev(yr)).cpu().numpy()
    xa_cu = ref_plan.sense_adjoint(to_dev(yr)).cpu().numpy()
    xa_o = onf.nufft_adjoint(yr.astype(np.complex128), maps.astype(np.complex128), traj, 1.25, 4)
    assert rel(xa, xa_o, "adjoint, own FFT passes vs oracle") < 1e-5
    assert rel(xa, xa_cu, "adjoint, own FFT passes vs cuFFT") < 2e-6
