// Batched reconstruction: many independent cases (each its own plan: image size, coils,
// trajectory, maps, regulariser, lambda) solved together.  The preconditioners are built case
// by case, each on its own stream; the power method's iterations (Sec. 6: 30 per case) and
// the PDHG iterations are each captured once into a CUDA graph holding every case on its own
// forked stream, so one graph launch advances all cases by one iteration and their kernels run
// concurrently on the GPU, with no per-case launches from the host.  Cases use the
// non-cooperative iteration (several cooperative grids would compete for co-residency).
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
};

namespace kp {
static void batch_drop_graph(kp_batch b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
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

kp_status kp_batch_destroy(kp_batch b) {
    if (!b) return KP_OK;
    cudaDeviceSynchronize();
    batch_drop_graph(b);
    batch_drop_pgraph(b);
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
    // (re)capture the all-case iteration graph when the regularisers, lambdas, data types or
    // any plan's buffers (trajectory, maps, schedule length) changed
    std::vector<int> kr(regs, regs + n), ky(n);
    std::vector<float> kl(lambdas, lambdas + n);
    std::vector<uint64_t> kg(n);
    for (int i = 0; i < n; ++i) {
        ky[i] = (int)y_types[i];
        kg[i] = b->plans[i]->graph_gen;
    }
    if (!b->exec || kr != b->key_reg || kl != b->key_lam || ky != b->key_yt || kg != b->key_gen) {
        batch_drop_graph(b);
        // capture issues nothing: each replay adds the kernels its part of the graph holds
        KP_TRY(capture_all(b, [&](int i, cudaStream_t s) {
            return pdhg_iteration_concurrent(b->plans[i], (int)regs[i], lambdas[i], s); }, &b->graph, &b->exec, b->per_replay));
        b->key_reg = kr;
        b->key_lam = kl;
        b->key_yt = ky;
        b->key_gen = kg;
    }
    for (int k = 0; k < iters; ++k) {
        KP_TRY_CUDA(cudaGraphLaunch(b->exec, st));
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
