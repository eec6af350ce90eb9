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


def test_forward_3d_ute_sampled():
    """3D centre-out radial 192^3 x 8 coils x 6.1M samples: the full-size launch checked on a
    sample of outputs, each against the exact oracle NUFFT restricted to those samples."""
    need_gpu()
    w, x, maps, traj = workload_problem("ute3d_192")
    C, M = maps.shape[0], traj.shape[0]
    plan = make_plan(x.shape, C, M, 1.25)
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    y = plan.sense_forward(to_dev(x)).cpu().numpy()
    idx = np.random.default_rng(0).choice(M, 300, replace=False)
    y_ref = onf.nufft_forward(x.astype(np.complex128), maps.astype(np.complex128), traj[idx], 1.25, 4)
    assert rel(y[:, idx], y_ref) < 1e-5


@pytest.mark.parametrize("storage,tol", [("bf16", 2.5e-3), ("fp16", 4e-4)])
def test_half_storage(storage, tol):
    need_gpu()
    from paper_1902_09657_gb300.api import to_storage
    x, maps, traj = random_problem((48, 40), 4, 3000, 7)
    y_ref = onf.nufft_forward(x.astype(np.complex128), maps.astype(np.complex128), traj, 1.25, 4)
    x_ref = onf.nufft_adjoint(y_ref, maps.astype(np.complex128), traj, 1.25, 4)
    plan = make_plan((48, 40), 4, 3000)
    plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
    y = plan.sense_forward(to_dev(x), storage=storage)
    yc = torch.view_as_complex(y.float().contiguous()).cpu().numpy()
    assert rel(yc, y_ref) < tol
    # maps stored in half precision, adjoint with half-storage input
    plan2 = make_plan((48, 40), 4, 3000)
    plan2.set_trajectory(to_dev(traj)).set_maps(to_storage(to_dev(maps), storage))
    xa = plan2.sense_adjoint(to_storage(to_dev(y_ref.astype(np.complex64)), storage)).cpu().numpy()
    assert rel(xa, x_ref) < 2 * tol


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
