// Batched reconstruction: many independent cases (each its own plan: image size, coils,
// trajectory, maps, regulariser, lambda) solved together.  The preconditioners are built case
// by case, each on its own stream; the power method's iterations (Sec. 6: 30 per case) replay
// one captured graph holding every case on its own forked stream.  The PDHG iteration has two
// layouts (kp_batch_set_form).  Phase form (2D l2 / l1-wavelet cases sharing the k-space and
// maps storage types):
// one kernel launch per phase over all cases (interpolation + dual step, split-tile clearing,
// spreading, primal step, each wavelet level, pre-step, counters), each block finding its case
// in a table of block offsets, with the cases' cuFFT transforms between the phases on forked
// streams, all captured into one graph.  Per-case form (the default, and whenever the phase
// form does not apply): each case's own iteration is captured on its own forked stream, so one
// case's FFTs overlap another's interpolation or spreading (measured faster on 64 uneven 2D
// cases: 7.1 against 8.7 ms per iteration of all cases).  Cases use the non-cooperative
// kernels (several cooperative grids would compete for co-residency).
#include "kp_internal.cuh"

#include <vector>

struct kp_batch_s {
    std::vector<kp_plan> plans;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t pgraph = nullptr;     // one power iteration of every case
    cudaGraphExec_t pexec = nullptr;
    std::vector<uint64_t> pkey_gen;
    std::vector<int64_t> pper_replay;
    std::vector<int> key_reg;
    std::vector<float> key_lam;
    std::vector<int> key_yt;
    std::vector<uint64_t> key_gen;   // plans' graph generations at capture
    std::vector<int64_t> per_replay;  // kernels each case adds per graph replay
    kp_batch_form form = KP_BATCH_PER_CASE;
    bool phase = false;               // the captured iteration graph is the phase form
    kp::BatchIter bi;                 // its batched launches
    int64_t phase_launches = 0;       // own kernels per phase-form replay
};

namespace kp {
static void batch_drop_graph(kp_batch b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Whether the phase form applies: every case 2D, l2 or l1-wavelet, with maps, and one k-space
// and one maps storage type across the batch.
static bool phase_form_ok(kp_batch b, const kp_cdtype* y_types, const kp_reg* regs) {
    if (b->form != KP_BATCH_PHASES) return false;
    const int n = (int)b->plans.size();
    for (int i = 0; i < n; ++i) {
        kp_plan p = b->plans[i];
        if (p->geo.D != 2 || p->unit_maps || (regs[i] != KP_REG_L2 && regs[i] != KP_REG_L1_WAVELET)) return false;
        if (y_types[i] != y_types[0] || p->maps_t != b->plans[0]->maps_t) return false;
    }
    return true;
}

// Issues issue(i, stream_i) for every case on forked streams of the capture stream and joins them.
template <typename F>
static kp_status fork_each(kp_batch b, F issue) {
    KP_TRY_CUDA(cudaEventRecord(b->fork, b->cap));
    for (int i = 0; i < (int)b->plans.size(); ++i) {
        KP_TRY_CUDA(cudaStreamWaitEvent(b->streams[i], b->fork, 0));
        KP_TRY(issue(i, b->streams[i]));
        KP_TRY_CUDA(cudaEventRecord(b->joins[i], b->streams[i]));
        KP_TRY_CUDA(cudaStreamWaitEvent(b->cap, b->joins[i], 0));
    }
    return KP_OK;
}

// One PDHG iteration of every case in phase form (issued on the capture stream).
static kp_status issue_phase_iteration(kp_batch b) {
    KP_TRY(fork_each(b, [&](int i, cudaStream_t s) { return fft_forward_only(b->plans[i], s); }));
    KP_TRY(batch_interp_launch(b->bi, b->cap));
    KP_TRY(batch_spread_launch(b->bi, b->cap));
    KP_TRY(fork_each(b, [&](int i, cudaStream_t s) { return fft_inverse_only(b->plans[i], s); }));
    KP_TRY(batch_primal_launch(b->bi, b->cap));
    KP_TRY(batch_wavelet_launch(b->bi, b->cap));
    return batch_pre_launch(b->bi, b->cap);
}

static kp_status capture_phase(kp_batch b, const std::vector<int>& regs, const std::vector<float>& lams) {
    batch_iter_free(b->bi);
    KP_TRY(batch_nufft_build(b->plans, regs, lams, b->bi));
    KP_TRY(batch_wavelet_build(b->plans, regs, lams, b->bi));
    int64_t nl = 1;                                                   // the counters
    for (const BatchPhase* ph : {&b->bi.interp, &b->bi.zero, &b->bi.spread, &b->bi.primal, &b->bi.pre})
        nl += ph->nblocks > 0;
    for (const auto& ph : b->bi.fwd) nl += ph.nblocks > 0;
    for (const auto& ph : b->bi.inv) nl += ph.nblocks > 0;
    b->phase_launches = nl;
    KP_TRY_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    const kp_status s = issue_phase_iteration(b);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (s != KP_OK) { if (g) cudaGraphDestroy(g); return s; }
    KP_TRY_CUDA(e);
    b->graph = g;
    KP_TRY_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
    b->bi.built = true;
    return KP_OK;
}

static void batch_drop_pgraph(kp_batch b) {
    if (b->pexec) cudaGraphExecDestroy(b->pexec);
    if (b->pgraph) cudaGraphDestroy(b->pgraph);
    b->pexec = nullptr;
    b->pgraph = nullptr;
}

// Captures `issue(i, stream)` for every case on its own forked stream of the capture stream.
template <typename F>
static kp_status capture_all(kp_batch b, F issue, cudaGraph_t* graph, cudaGraphExec_t* exec, std::vector<int64_t>& per) {
    const int n = (int)b->plans.size();
    std::vector<int64_t> before(n);
    for (int i = 0; i < n; ++i) before[i] = b->plans[i]->launches;
    KP_TRY_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    kp_status s = KP_OK;
    if (cudaEventRecord(b->fork, b->cap) != cudaSuccess) s = KP_ECUDA;
    for (int i = 0; s == KP_OK && i < n; ++i) {
        if (cudaStreamWaitEvent(b->streams[i], b->fork, 0) != cudaSuccess) { s = KP_ECUDA; break; }
        s = issue(i, b->streams[i]);
        if (s == KP_OK && (cudaEventRecord(b->joins[i], b->streams[i]) != cudaSuccess ||
                           cudaStreamWaitEvent(b->cap, b->joins[i], 0) != cudaSuccess))
            s = KP_ECUDA;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    per.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        per[i] = b->plans[i]->launches - before[i];
        b->plans[i]->launches = before[i];
    }
    if (s != KP_OK) { if (g) cudaGraphDestroy(g); return s; }
    KP_TRY_CUDA(e);
    *graph = g;
    KP_TRY_CUDA(cudaGraphInstantiate(exec, g, 0));
    return KP_OK;
}
}  // namespace kp

using namespace kp;

extern "C" {

kp_status kp_batch_create(kp_batch* out, kp_plan* plans, int ncases) {
    KP_RANGE("kp_batch_create");
    if (!out || !plans || ncases < 1) { set_error("null argument or ncases < 1"); return KP_EINVAL; }
    *out = nullptr;
    kp_batch b = new (std::nothrow) kp_batch_s();
    if (!b) { set_error("host allocation failed"); return KP_ENOMEM; }
    for (int i = 0; i < ncases; ++i) {
        if (!plans[i]) { delete b; set_error("null plan in batch"); return KP_EINVAL; }
        b->plans.push_back(plans[i]);
    }
    b->streams.assign(ncases, nullptr);
    b->joins.assign(ncases, nullptr);
    kp_status s = KP_OK;
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
        s = KP_ECUDA;
    for (int i = 0; s == KP_OK && i < ncases; ++i) {
        if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming) != cudaSuccess)
            s = KP_ECUDA;
    }
    if (s != KP_OK) {
        kp_batch_destroy(b);
        set_error("stream or event creation failed");
        return s;
    }
    *out = b;
    return KP_OK;
}

kp_status kp_batch_set_form(kp_batch b, kp_batch_form form) {
    if (!b) { set_error("null batch"); return KP_EINVAL; }
    if (form != KP_BATCH_PER_CASE && form != KP_BATCH_PHASES) { set_error("unknown batch form"); return KP_EINVAL; }
    b->form = form;
    return KP_OK;
}

kp_status kp_batch_destroy(kp_batch b) {
    if (!b) return KP_OK;
    cudaDeviceSynchronize();
    batch_drop_graph(b);
    batch_drop_pgraph(b);
    batch_iter_free(b->bi);
    for (auto s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (auto e : b->joins)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return KP_OK;
}

kp_status kp_batch_solve(kp_batch b, const void* const* y_devs, const kp_cdtype* y_types, const float* const* p_devs,
                         const kp_reg* regs, const float* lambdas, int iters, void* const* x_devs, void* stream) {
    KP_RANGE("kp_batch_solve");
    if (!b || !y_devs || !y_types || !regs || !lambdas || !x_devs) { set_error("null argument"); return KP_EINVAL; }
    if (iters < 0) { set_error("iters must be >= 0"); return KP_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)b->plans.size();
    for (int i = 0; i < n; ++i) {
        kp_plan p = b->plans[i];
        if (!p->traj_set || !p->maps_set) { set_error("every plan needs a trajectory and maps"); return KP_EINVAL; }
        if (regs[i] != KP_REG_L2 && regs[i] != KP_REG_L1_WAVELET && regs[i] != KP_REG_TV) { set_error("bad regulariser"); return KP_EINVAL; }
        if (regs[i] == KP_REG_L1_WAVELET && p->P.wavelet_levels < 1) { set_error("l1-wavelet case without levels"); return KP_EINVAL; }
    }
    // the phase form spreads every case with the per-tile lists of the single-pass kernels,
    // which a plan tuned to a two-phase variant has not built for its trajectory
    const bool phase = phase_form_ok(b, y_types, regs);
    if (phase)
        for (int i = 0; i < n; ++i)
            if (b->plans[i]->lists_version != b->plans[i]->traj_version) KP_TRY(build_spread_lists(b->plans[i], st));
    // per-case set-up before lambda_max (measurements, preconditioner, min p, start vector),
    // each case on its own stream so the cases' set-up kernels overlap
    KP_TRY_CUDA(cudaEventRecord(b->fork, st));
    for (int i = 0; i < n; ++i) {
        kp_plan p = b->plans[i];
        KP_TRY_CUDA(cudaStreamWaitEvent(b->streams[i], b->fork, 0));
        KP_TRY(solve_setup_a(p, y_devs[i], y_types[i], p_devs ? p_devs[i] : nullptr, std::max(iters, 1),
                             b->streams[i], nullptr));
        KP_TRY(fill_image(p->d_z, p->geo.N, make_float2(1.f, 0.f), b->streams[i]));
        p->launches += 1;
        KP_TRY(power_begin(p, b->streams[i]));
        KP_TRY(power_step(p, p->d_ps, true, b->streams[i]));       // first iteration reads d_z
        KP_TRY_CUDA(cudaEventRecord(b->joins[i], b->streams[i]));
        KP_TRY_CUDA(cudaStreamWaitEvent(st, b->joins[i], 0));
    }
    // the other 29 power iterations of every case: one graph replayed on the caller's stream
    {
        std::vector<uint64_t> kg(n);
        for (int i = 0; i < n; ++i) kg[i] = b->plans[i]->graph_gen;
        if (!b->pexec || kg != b->pkey_gen) {
            batch_drop_pgraph(b);
            KP_TRY(capture_all(b, [&](int i, cudaStream_t s) { return power_step(b->plans[i], b->plans[i]->d_ps, false, s); },
                               &b->pgraph, &b->pexec, b->pper_replay));
            b->pkey_gen = kg;
        }
        for (int k = 1; k < 30; ++k) {
            KP_TRY_CUDA(cudaGraphLaunch(b->pexec, st));
            for (int i = 0; i < n; ++i) b->plans[i]->launches += b->pper_replay[i];
        }
    }
    // lambda_max, the schedule, zero iterates, per case
    KP_TRY_CUDA(cudaEventRecord(b->fork, st));
    for (int i = 0; i < n; ++i) {
        kp_plan p = b->plans[i];
        KP_TRY_CUDA(cudaStreamWaitEvent(b->streams[i], b->fork, 0));
        KP_TRY(power_end(p, b->streams[i]));
        KP_TRY(solve_setup_b(p, std::max(iters, 1), b->streams[i], (int)regs[i], nullptr));
        KP_TRY_CUDA(cudaEventRecord(b->joins[i], b->streams[i]));
        KP_TRY_CUDA(cudaStreamWaitEvent(st, b->joins[i], 0));
    }
    // (re)capture the all-case iteration graph when the form, the regularisers, lambdas, data
    // types or any plan's buffers (trajectory, maps, schedule length) changed
    std::vector<int> kr(regs, regs + n), ky(n);
    std::vector<float> kl(lambdas, lambdas + n);
    std::vector<uint64_t> kg(n);
    for (int i = 0; i < n; ++i) {
        ky[i] = (int)y_types[i];
        kg[i] = b->plans[i]->graph_gen;
    }
    if (!b->exec || phase != b->phase || kr != b->key_reg || kl != b->key_lam || ky != b->key_yt || kg != b->key_gen) {
        batch_drop_graph(b);
        if (phase) {
            KP_TRY(capture_phase(b, kr, kl));
        } else {
            // capture issues nothing: each replay adds the kernels its part of the graph holds
            KP_TRY(capture_all(b, [&](int i, cudaStream_t s) {
                return pdhg_iteration_concurrent(b->plans[i], (int)regs[i], lambdas[i], s); }, &b->graph, &b->exec, b->per_replay));
        }
        b->phase = phase;
        b->key_reg = kr;
        b->key_lam = kl;
        b->key_yt = ky;
        b->key_gen = kg;
    }
    for (int k = 0; k < iters; ++k) {
        KP_TRY_CUDA(cudaGraphLaunch(b->exec, st));
        if (phase) b->plans[0]->launches += b->phase_launches;
        else
            for (int i = 0; i < n; ++i) b->plans[i]->launches += b->per_replay[i];
    }
    for (int i = 0; i < n; ++i) {
        kp_plan p = b->plans[i];
        KP_TRY_CUDA(cudaMemcpyAsync(x_devs[i], p->d_x, p->geo.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    }
    std::vector<int> flags(KP_NFLAGS * (size_t)n);
    for (int i = 0; i < n; ++i)
        KP_TRY_CUDA(cudaMemcpyAsync(&flags[KP_NFLAGS * (size_t)i], b->plans[i]->d_flag, KP_NFLAGS * sizeof(int),
                                    cudaMemcpyDeviceToHost, st));
    KP_TRY_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i) {
        const int* f = &flags[KP_NFLAGS * (size_t)i];
        if (f[KP_FLAG_P_BAD] != 0 || f[KP_FLAG_SCHED_BAD] != 0) {
            set_error("case " + std::to_string(i) + ": preconditioner or lambda_max not positive and finite");
            return KP_EINVAL;
        }
        if (f[KP_FLAG_TIMEOUT] != 0) {
            for (int j = i + 1; j < n; ++j)      // consume the later cases' reports too
                if (flags[KP_NFLAGS * (size_t)j + KP_FLAG_TIMEOUT] != 0)
                    KP_TRY_CUDA(cudaMemsetAsync(b->plans[j]->d_flag + KP_FLAG_TIMEOUT, 0, sizeof(int), st));
            return report_timeout(b->plans[i], st, ("case " + std::to_string(i) + ": a bounded device wait gave up").c_str());
        }
    }
    return KP_OK;
}

}  // extern "C"
