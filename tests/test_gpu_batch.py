"""Batched reconstruction (kp_batch): many independent cases, each with its own image size,
coil count, trajectory, regulariser and lambda, advanced together by one CUDA graph per
Sec. 4.1 iteration.  Each case must match (a) the float64 oracle's PDHG from the same p and
lambda_max and (b) the single-case solver kp_pdhg_solve on the same plan."""
import numpy as np
import pytest

from oracle import nufft as onf, precond as opc, solvers as osv
from tests.gpu_util import need_gpu, rel, simulate, to_dev, make_plan
import synth

pytestmark = pytest.mark.gpu


def _case(i, n, C, kind, spokes, reg, levels):
    if kind == "radial":
        targs = dict(n_spokes=spokes, n_readout=2 * n, kmax=n / 2.0)
    else:
        targs = dict(n_interleaves=spokes, n_samples=2 * n, kmax=n / 2.0)
    return synth.Workload(f"b{i}", (n, n), C, 1.25, 4, reg, 1e-3, 20, levels, kind, targs, seed=500 + i)


# uneven sizes, both trajectory kinds, both regularisers; 48 has a ragged tile, 40 needs a
# different tile size than 64
CASES = [(0, 64, 4, "spiral", 6, "l1_wavelet", 3), (1, 48, 3, "radial", 40, "l2", 0),
         (2, 40, 5, "radial", 24, "l1_wavelet", 2), (3, 32, 2, "spiral", 4, "l2", 0)]


def _setup(cases):
    plans, ys, ps, Ls, lams, oracle_in = [], [], [], [], [], []
    for spec in cases:
        w = _case(*spec)
        x, maps, traj = w.phantom(), w.maps(), w.traj()
        y = simulate(w, x, maps, traj)
        m = maps.astype(np.complex128)
        A = lambda v, m=m, traj=traj: onf.nufft_forward(v, m, traj, 1.25, 4)
        AH = lambda u, m=m, traj=traj: onf.nufft_adjoint(u, m, traj, 1.25, 4)
        p = opc.mc_precond_fast(m, traj, 1.25, 4)
        L, _ = osv.power_method(A, AH, p, x.shape, iters=30)
        lam = 1e-3
        if w.reg == "l1_wavelet":
            lam = lam * float(np.abs(AH(y.astype(np.complex128))).max())
        plan = make_plan(x.shape, maps.shape[0], traj.shape[0], levels=w.wavelet_levels)
        plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
        plans.append(plan)
        ys.append(y)
        ps.append(p)
        Ls.append(L)
        lams.append(lam)
        oracle_in.append((w, A, AH, x.shape))
    return plans, ys, ps, Ls, lams, oracle_in


def test_batch_matches_oracle_and_single_solves():
    need_gpu()
    from paper_1902_09657_gb300.api import Batch
    plans, ys, ps, Ls, lams, oin = _setup(CASES)
    iters = 40
    regs = [c[5] for c in CASES]
    batch = Batch(plans)
    yd = [to_dev(y) for y in ys]
    pd = [to_dev(p.astype(np.float32)) for p in ps]
    xs = batch.solve(yd, pd, regs, lams, iters)
    for i, (w, A, AH, shape) in enumerate(oin):
        x_ref, _, _, _ = osv.pdhg(A, AH, ys[i], ps[i], shape, regs[i], lams[i], iters, Ls[i],
                                  levels=w.wavelet_levels)
        # the batch runs its own power method (float32 operators, float64 norms)
        assert rel(xs[i].cpu().numpy(), x_ref, f"case {i} vs oracle") < 1e-5, i
        xg, _, st = plans[i].pdhg_solve(yd[i], pd[i], regs[i], lams[i], iters)
        assert rel(xs[i].cpu().numpy(), xg.cpu().numpy(), f"case {i} vs single solve") < 2e-6, i
    batch.close()


def test_batch_graph_reuse_and_recapture():
    """A second solve replays the cached graph (same result); a new lambda or regulariser
    re-captures; a changed trajectory (new tiles and buffers) re-captures too."""
    need_gpu()
    from paper_1902_09657_gb300.api import Batch
    cases = CASES[1:3]
    plans, ys, ps, Ls, lams, oin = _setup(cases)
    regs = [c[5] for c in cases]
    batch = Batch(plans)
    yd = [to_dev(y) for y in ys]
    xa = batch.solve(yd, None, regs, lams, 15)
    xb = batch.solve(yd, None, regs, lams, 15)
    for a, b in zip(xa, xb):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-6
    lams2 = [2 * v for v in lams]
    xc = batch.solve(yd, None, regs, lams2, 15)
    for i in range(2):
        xg, _, _ = plans[i].pdhg_solve(yd[i], None, regs[i], lams2[i], 15)
        assert rel(xc[i].cpu().numpy(), xg.cpu().numpy()) < 2e-6
    # new trajectory on case 0 (same sample count): the batch must not replay stale buffers
    w = _case(*cases[0])
    rng = np.random.default_rng(7)
    traj2 = (w.traj() + rng.uniform(-0.3, 0.3, w.traj().shape)).clip(-w.img_shape[0] / 2, w.img_shape[0] / 2 - 1e-3)
    plans[0].set_trajectory(to_dev(traj2.astype(np.float32)))
    xd = batch.solve(yd, None, regs, lams, 15)
    xg, _, _ = plans[0].pdhg_solve(yd[0], None, regs[0], lams[0], 15)
    assert rel(xd[0].cpu().numpy(), xg.cpu().numpy()) < 2e-6
    assert rel(xd[1].cpu().numpy(), xa[1].cpu().numpy()) < 1e-6
    batch.close()


def test_batch_launch_count_and_bad_inputs():
    need_gpu()
    from paper_1902_09657_gb300.api import Batch
    from paper_1902_09657_gb300._lib import KpError
    cases = CASES[:2]
    plans, ys, ps, Ls, lams, oin = _setup(cases)
    regs = [c[5] for c in cases]
    batch = Batch(plans)
    yd = [to_dev(y) for y in ys]
    batch.solve(yd, None, regs, lams, 3)
    before = [p.launch_count() for p in plans]
    batch.solve(yd, None, regs, lams, 7)
    grown = [p.launch_count() - b for p, b in zip(plans, before)]
    assert all(g > 0 for g in grown) and sum(grown) > 7   # per-iteration kernels are counted on replay
    with pytest.raises(KpError):
        batch.solve(yd, None, ["l1_wavelet", "l1_wavelet"], lams, 3)   # case 1 has no wavelet levels
    bad = np.ones(ps[0].shape, np.float32)
    bad[0, 5] = 0.0
    with pytest.raises(KpError):
        batch.solve(yd, [to_dev(bad), None], regs, lams, 3)
    batch.close()


def _iteration_launches(batch, plans, yd, regs, lams):
    """Own kernels one batched PDHG iteration adds (two solves that differ by 7 iterations)."""
    def grown(iters):
        before = sum(p.launch_count() for p in plans)
        xs = batch.solve(yd, None, regs, lams, iters)
        return sum(p.launch_count() for p in plans) - before, xs
    grown(3)                                   # capture
    d3, _ = grown(3)
    d10, xs = grown(10)
    assert (d10 - d3) % 7 == 0
    return (d10 - d3) // 7, xs


def test_batch_phase_form():
    """2D l2 / l1-wavelet cases in the phase form: one launch per phase over all cases
    (interpolation, split clearing, spreading, primal step, each wavelet level, pre-step,
    counters), so the own kernels per iteration do not grow with the number of cases; the
    results equal the per-case form's and the oracle's."""
    need_gpu()
    from paper_1902_09657_gb300.api import Batch
    plans, ys, ps, Ls, lams, oin = _setup(CASES)
    regs = [c[5] for c in CASES]
    yd = [to_dev(y) for y in ys]
    pd = [to_dev(p.astype(np.float32)) for p in ps]
    batch = Batch(plans, form="phases")
    per_phase, xs_phase = _iteration_launches(batch, plans, yd, regs, lams)
    lmax = max(c[6] for c in CASES)
    assert per_phase <= 7 + 2 * lmax
    batch.set_form("per_case")
    per_case, xs_case = _iteration_launches(batch, plans, yd, regs, lams)
    assert per_case > per_phase
    for i in range(len(CASES)):
        assert rel(xs_phase[i].cpu().numpy(), xs_case[i].cpu().numpy(), f"case {i} phase vs per-case form") < 2e-6, i
    batch.set_form("phases")
    iters = 40
    xs = batch.solve(yd, pd, regs, lams, iters)
    for i, (w, A, AH, shape) in enumerate(oin):
        x_ref, _, _, _ = osv.pdhg(A, AH, ys[i], ps[i], shape, regs[i], lams[i], iters, Ls[i], levels=w.wavelet_levels)
        assert rel(xs[i].cpu().numpy(), x_ref, f"case {i} phase form vs oracle") < 1e-5, i
    batch.close()


def test_batch_uneven_workload_cases():
    """The first cases of the 64-case uneven workload (image 96..320, 4..32 coils): batched
    results equal the per-case solver's."""
    need_gpu()
    from paper_1902_09657_gb300.api import Batch, Plan
    import torch
    cases = synth.batched_cases(6)
    plans, yd, lams = [], [], []
    g = torch.Generator(device="cuda").manual_seed(3)
    for w in cases:
        traj = w.traj()
        plan = Plan(w.img_shape, w.ncoils, traj.shape[0], wavelet_levels=w.wavelet_levels)
        plan.set_trajectory(to_dev(traj)).set_maps(to_dev(w.maps()))
        y = torch.randn((w.ncoils, traj.shape[0]), dtype=torch.complex64, device="cuda", generator=g)
        plans.append(plan)
        yd.append(y)
        lams.append(1e-3 * (float(plan.sense_adjoint(y).abs().max()) if w.reg == "l1_wavelet" else 1.0))
    regs = [w.reg for w in cases]
    xs = Batch(plans).solve(yd, None, regs, lams, 20)
    for i in range(len(cases)):
        xg, _, _ = plans[i].pdhg_solve(yd[i], None, regs[i], lams[i], 20)
        assert rel(xs[i].cpu().numpy(), xg.cpu().numpy()) < 2e-6, i


def test_batch_tv_case():
    """A TV case (Sec. 4.2) next to an l2 case in one batch: each equals its single-plan solve."""
    need_gpu()
    from paper_1902_09657_gb300.api import Batch
    cases = [(0, 64, 4, "spiral", 6, "tv", 0), (1, 48, 3, "radial", 40, "l2", 0)]
    plans, ys, ps, Ls, lams, oin = _setup(cases)
    regs = [c[5] for c in cases]
    yd = [to_dev(y) for y in ys]
    xs = Batch(plans).solve(yd, None, regs, lams, 20)
    for i in range(len(cases)):
        xg, _, _ = plans[i].pdhg_solve(yd[i], None, regs[i], lams[i], 20)
        assert rel(xs[i].cpu().numpy(), xg.cpu().numpy()) < 2e-6, i


def test_batch_uneven_bf16_kspace_against_oracle():
    """Three cases of the uneven 64-case workload (160^2 x 9 coils l1-wavelet radial, 256^2 x 4
    coils l2 radial, 96^2 x 6 coils l2 spiral) with their measurements stored in bf16, solved
    together for 20 iterations; each case's preconditioner and lambda_max are computed by the
    batch.  Against the float64 oracle's whole chain on the stored (rounded) measurements:
    1e-5; against the oracle on the unrounded measurements: 2e-3 (one bf16 rounding)."""
    need_gpu()
    import torch
    from paper_1902_09657_gb300.api import Batch, Plan, to_storage
    from tests.gpu_util import rounded
    allc = synth.batched_cases(64)
    cases = [allc[3], allc[4], allc[7]]
    plans, yd, lams, ref = [], [], [], []
    for w in cases:
        x, maps, traj = w.phantom(), w.maps(), w.traj()
        y = simulate(w, x, maps, traj)
        ys = to_storage(to_dev(y), "bf16")
        m = maps.astype(np.complex128)
        A = lambda v, m=m, traj=traj: onf.nufft_forward(v, m, traj, 1.25, 4)
        AH = lambda u, m=m, traj=traj: onf.nufft_adjoint(u, m, traj, 1.25, 4)
        p = opc.mc_precond_fast(m, traj, 1.25, 4)
        L, _ = osv.power_method(A, AH, p, x.shape, iters=30)
        y_st = rounded(ys).reshape(y.shape)
        lam = 1e-3
        if w.reg == "l1_wavelet":
            lam = lam * float(np.abs(AH(y_st)).max())
        x_st = osv.pdhg(A, AH, y_st, p, x.shape, w.reg, lam, 20, L, levels=w.wavelet_levels)[0]
        x_unr = osv.pdhg(A, AH, y, p, x.shape, w.reg, lam, 20, L, levels=w.wavelet_levels)[0]
        plan = Plan(w.img_shape, w.ncoils, traj.shape[0], wavelet_levels=w.wavelet_levels)
        plan.set_trajectory(to_dev(traj)).set_maps(to_dev(maps))
        plans.append(plan)
        yd.append(ys)
        lams.append(lam)
        ref.append((x_st, x_unr))
    xs = Batch(plans).solve(yd, None, [w.reg for w in cases], lams, 20)
    for i, (x_st, x_unr) in enumerate(ref):
        xg = xs[i].cpu().numpy()
        assert rel(xg, x_st, f"case {i} vs oracle on stored y") < 1e-5, i
        assert rel(xg, x_unr, f"case {i} storage error") < 2e-3, i
