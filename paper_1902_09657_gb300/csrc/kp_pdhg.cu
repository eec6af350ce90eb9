// Preconditioned PDHG (Sec. 4.1), the power method for lambda_max(P A A^H) (Sec. 6) and the
// periodised Daubechies-4 wavelet W used by the l1 prox (Sec. 2, Sec. 6).
//
// One PDHG iteration = FFT of the forward grid -> interpolation + dual update -> spreading ->
// inverse FFT -> fused primal kernel (adjoint combine, z = x - tau A^H u, l2 or l1-wavelet
// prox, extrapolation, the next iteration's forward pre-step, iteration counter).  The step
// sizes sigma_k, tau_k, theta_k are computed on the device in float64 from lambda_max and
// min p, so one captured CUDA graph replays every iteration.
#include "kp_internal.cuh"

#include <cstdlib>

#include <cmath>
#include <complex>
#include <vector>

namespace kp {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ================================================================ Daubechies-4 filter
// Extremal-phase Daubechies scaling filter with 4 vanishing moments, by spectral
// factorisation: the roots y_r of P(y) = 1 + 4y + 10y^2 + 20y^3 map to z_r with
// z + 1/z = 2 - 4 y_r, |z_r| < 1; H(z) ~ (1 + z^{-1})^4 prod_r (1 - z_r z^{-1}), sum h = sqrt(2).
void daubechies4(float hout[8]) {
    using cd = std::complex<double>;
    const double pc[4] = {1.0, 4.0, 10.0, 20.0};          // ascending powers of y
    // Durand-Kerner iteration on the monic cubic y^3 + (10/20) y^2 + (4/20) y + 1/20.
    auto P = [&](cd y) { return ((y + pc[2] / pc[3]) * y + pc[1] / pc[3]) * y + pc[0] / pc[3]; };
    cd r[3] = {cd(0.4, 0.9), cd(0.4, 0.9) * cd(0.4, 0.9), cd(0.4, 0.9) * cd(0.4, 0.9) * cd(0.4, 0.9)};
    for (int it = 0; it < 500; ++it) {
        for (int i = 0; i < 3; ++i) {
            cd den = 1.0;
            for (int j = 0; j < 3; ++j)
                if (j != i) den *= r[i] - r[j];
            r[i] -= P(r[i]) / den;
        }
    }
    std::vector<cd> poly = {1.0};
    auto mul = [&](cd a0, cd a1) {           // poly *= (a0 + a1 z^{-1})
        std::vector<cd> out(poly.size() + 1, 0.0);
        for (size_t k = 0; k < poly.size(); ++k) {
            out[k] += a0 * poly[k];
            out[k + 1] += a1 * poly[k];
        }
        poly.swap(out);
    };
    for (int k = 0; k < 4; ++k) mul(1.0, 1.0);
    for (int i = 0; i < 3; ++i) {
        cd b = 2.0 - 4.0 * r[i];
        cd disc = std::sqrt(b * b - 4.0);
        cd z1 = (b + disc) / 2.0, z2 = (b - disc) / 2.0;
        cd z = std::abs(z1) < 1.0 ? z1 : z2;
        mul(1.0, -z);
    }
    double sum = 0;
    for (int k = 0; k < 8; ++k) sum += poly[k].real();
    for (int k = 0; k < 8; ++k) hout[k] = (float)(poly[k].real() * std::sqrt(2.0) / sum);
}

// ================================================================ reductions and small kernels
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// out += sum of f(i) over i < n  (blocks of 256 threads)
template <typename F>
__device__ __forceinline__ void block_sum_to(double v, double* out) {
    __shared__ double ws[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) atomicAdd(out, v);
    }
}

__global__ void k_norm2(const float2* __restrict__ x, int64_t n, double* __restrict__ out) {
    double s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float2 v = x[i];
        s += (double)v.x * v.x + (double)v.y * v.y;
    }
    block_sum_to<int>(s, out);
}

__global__ void k_sumabs(const float2* __restrict__ x, int64_t n, double* __restrict__ out) {
    double s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float2 v = x[i];
        s += sqrt((double)v.x * v.x + (double)v.y * v.y);
    }
    block_sum_to<int>(s, out);
}

template <typename YT>
__global__ void k_resid2(const float2* __restrict__ a, const YT* __restrict__ y, int64_t n, double* __restrict__ out) {
    double s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float2 v = a[i];
        float2 w = ldc<YT>(y, i);
        double dx = (double)v.x - w.x, dy = (double)v.y - w.y;
        s += dx * dx + dy * dy;
    }
    block_sum_to<int>(s, out);
}

// min over positive p (as int bits) and count of non-positive / non-finite entries
__global__ void k_pmin(const float* __restrict__ p, int64_t n, int* __restrict__ minbits, int* __restrict__ bad) {
    int m = 0x7f7fffff;
    int nb = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float v = p[i];
        if (!(v > 0.f) || !isfinite(v)) ++nb;
        else m = min(m, __float_as_int(v));
    }
    atomicMin(minbits, m);
    if (nb) atomicAdd(bad, nb);
}

// ||x||^2 added into *out and, in the same launch, the split spreading tiles of grid2 cleared
// for the next spread (the previous kernel was the last to read grid2).
template <int D>
__global__ void k_norm2_clear(const float2* __restrict__ x, int64_t n, double* __restrict__ out,
                              const int* __restrict__ split, int n_split, Geom geo, Tiles tl, float2* __restrict__ grid2) {
    double s = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float2 v = x[i];
        s += (double)v.x * v.x + (double)v.y * v.y;
    }
    block_sum_to<int>(s, out);
    for (int t = blockIdx.x; t < n_split; t += gridDim.x) {    // one split tile per block pass
        int r = split[t], o[MAXD], e[MAXD], P = 1;
        for (int d = D - 1; d >= 0; --d) {
            const int tc = r % tl.nt[d];
            r /= tl.nt[d];
            o[d] = tc * tl.ts[d];
            e[d] = min(tl.ts[d], geo.g[d] - o[d]);
        }
        for (int d = 0; d < D; ++d) P *= e[d];
        for (int i = threadIdx.x; i < geo.C * P; i += blockDim.x) {
            const int c = i / P;
            int rr = i - c * P, lidx[MAXD];
            for (int d = D - 1; d >= 0; --d) { lidx[d] = rr % e[d]; rr /= e[d]; }
            int64_t gflat = 0;
            for (int d = 0; d < D; ++d) gflat = gflat * geo.g[d] + tunshift(o[d] + lidx[d], tl.sh[d], geo.g[d]);
            grid2[(size_t)c * geo.G + gflat] = make_float2(0.f, 0.f);
        }
    }
}

__global__ void k_store_sqrt(const double* __restrict__ n2, double* __restrict__ out) { *out = sqrt(*n2); }

// Step sizes (Sec. 4.1): sigma_0 = 1, tau_0 = 1/L, theta_k = 1/(1 + 2 sigma_k pmin),
// sigma_{k+1} = theta_k sigma_k, tau_{k+1} = tau_k / theta_k; float64 recursion.
// schedd: [0] L, [1] pmin (written here from minbits), [2] sigma_last, [3] tau_last.
// tv_d > 0: the fixed steps of Sec. 4.2 for TV in tv_d dimensions, sigma = theta = 1 and
// tau = 1/(L + lambda_max(G G^H)) with lambda_max(G G^H) = 4 tv_d.
__global__ void k_schedule(double* __restrict__ schedd, const int* __restrict__ minbits, int iters,
                           float* __restrict__ sched, int* __restrict__ flag, int tv_d) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double L = schedd[0];
    const double pmin = minbits ? (double)__int_as_float(*minbits) : schedd[1];
    schedd[1] = pmin;
    if (!(L > 0) || !isfinite(L) || !(pmin > 0) || !isfinite(pmin)) {
        flag[0] = 1;
        for (int k = 0; k < iters; ++k) { sched[3 * k] = 0.f; sched[3 * k + 1] = 0.f; sched[3 * k + 2] = 0.f; }
        return;
    }
    if (tv_d > 0) {
        const double tau = 1.0 / (L + 4.0 * tv_d);
        for (int k = 0; k < iters; ++k) {
            sched[3 * k] = 1.f;
            sched[3 * k + 1] = (float)tau;
            sched[3 * k + 2] = 1.f;
        }
        schedd[2] = 1.0;
        schedd[3] = tau;
        return;
    }
    double sig = 1.0, tau = 1.0 / L;
    for (int k = 0; k < iters; ++k) {
        const double th = 1.0 / (1.0 + 2.0 * sig * pmin);
        sched[3 * k] = (float)sig;
        sched[3 * k + 1] = (float)tau;
        sched[3 * k + 2] = (float)th;
        sig *= th;
        tau /= th;
    }
    schedd[2] = sig;
    schedd[3] = tau;
}

__global__ void k_advance(int* iter) { *iter += 1; }

// out[c][perm[s]] = in[c][s]: a sorted-order k-space array back to the trajectory's order
__global__ void k_unpermute_c64(const float2* __restrict__ in, float2* __restrict__ out, const int* __restrict__ perm,
                                int64_t M, int C) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const int64_t o = perm[s];
    for (int c = 0; c < C; ++c) out[(size_t)c * M + o] = in[(size_t)c * M + s];
}

__global__ void k_set_int(int* p, int v) { *p = v; }

__global__ void k_set_double(double* p, double v) { *p = v; }

// flag = 1 if any of the n complex values is a NaN or an Inf
__global__ void k_nonfinite(const float2* __restrict__ x, int64_t n, int* __restrict__ flag) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = x[i];
        bad |= !isfinite(v.x) || !isfinite(v.y);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

template <typename T>
__global__ void k_permute(const T* __restrict__ in, T* __restrict__ out, const int* __restrict__ perm, int64_t M, int C) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const int64_t o = perm[s];
    for (int c = 0; c < C; ++c) out[(size_t)c * M + s] = in[(size_t)c * M + o];
}

// ================================================================ host drivers
static kp_status reduce_norm2(kp_plan p, const float2* x, int64_t n, double* out, cudaStream_t st) {
    KP_TRY_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
    k_norm2<<<(unsigned)std::min<int64_t>(nblk(n, 256), 1216), 256, 0, st>>>(x, n, out);
    KP_LAUNCH_CHECK();
    p->launches += 1;
    return KP_OK;
}

// Power method on A^H P A (Sec. 6: 30 iterations) using the sorted p in d_ps (or none).
// Start vector in d_z (unnormalised); result L in d_schedd[0].  Each iteration applies
// A^H P A to w / ||w|| without forming it: the forward pre-step reads w and the interpolation
// divides by ||w||, taken from the device (the same vector up to rounding order); the norm
// kernel also clears the split spreading tiles for the next spread.  L = ||w|| of the last
// iteration, w = A^H P A v with v of unit norm.  In three parts so that a batch can capture the
// middle one for all its cases in one graph: begin (norm of the start vector), step (one
// iteration; the first reads d_z, later ones d_w) and end (L = sqrt of the last norm).
kp_status power_begin(kp_plan p, cudaStream_t st) {
    KP_TRY(zero_split_only(p, st));
    return reduce_norm2(p, p->d_z, p->geo.N, p->d_red, st);
}

kp_status power_step(kp_plan p, const float* ps_sorted, bool first, cudaStream_t st) {
    const Geom& g = p->geo;
    const int n_split = p->spread_variant >= 10 ? 0 : (int)p->n_split;   // 10-12 store every point
    const unsigned nb = (unsigned)std::min<int64_t>(nblk(g.N, 256), 1216);
    KP_TRY(forward_scaled(p, first ? p->d_z : p->d_w, p->d_kt, ps_sorted, st, p->d_red));
    KP_TRY(adjoint_to_grid(p, p->d_kt, KP_C64, nullptr, st, /*splits_zeroed=*/true));
    KP_TRY(grid_to_image(p, p->d_w, st));
    KP_TRY_CUDA(cudaMemsetAsync(p->d_red, 0, sizeof(double), st));
    if (g.D == 2)
        k_norm2_clear<2><<<nb, 256, 0, st>>>(p->d_w, g.N, p->d_red, p->d_split, n_split, g, p->tiles, p->d_grid2);
    else
        k_norm2_clear<3><<<nb, 256, 0, st>>>(p->d_w, g.N, p->d_red, p->d_split, n_split, g, p->tiles, p->d_grid2);
    KP_LAUNCH_CHECK();
    p->launches += 1;
    return KP_OK;
}

kp_status power_end(kp_plan p, cudaStream_t st) {
    k_store_sqrt<<<1, 1, 0, st>>>(p->d_red, p->d_schedd);
    KP_LAUNCH_CHECK();
    p->launches += 1;
    return KP_OK;
}

static kp_status power_method(kp_plan p, const float* ps_sorted, int iters, cudaStream_t st) {
    KP_PHASE("power_method");
    KP_TRY(power_begin(p, st));
    for (int it = 0; it < iters; ++it) KP_TRY(power_step(p, ps_sorted, it == 0, st));
    return power_end(p, st);
}

// Whether the primal step runs as separate kernels (combine + step, wavelet levels or pre-step,
// counter) instead of one persistent cooperative kernel (one CTA per SM, grid barriers between
// the phases).  KPDHG_PRIMAL=levels selects the separate kernels; the fused kernel is the default
// (3D UTE 192^3 x 8 coils, l1: 1.62 ms against 2.15 ms per iteration).
static bool levels_primal(kp_plan p) {
    const char* e = std::getenv("KPDHG_PRIMAL");
    if (e && std::string(e) == "levels") return true;
    if (e && std::string(e) == "fused") return false;
    (void)p;
    return false;
}

// One PDHG iteration (Sec. 4.1) from the forward grid of xbar already in d_grid:
// FFT -> interpolation + dual update -> spreading + inverse FFT -> fused primal step
// (adjoint combine, prox, extrapolation, next forward pre-step, counter).
static kp_status issue_iteration(kp_plan p, int reg, float lambda, cudaStream_t st) {
    KP_TRY(fft_forward_only(p, st));
    KP_TRY(interp_dual_only(p, st));
    if (reg == KP_REG_TV) {
        // Sec. 4.2: spreading (it clears its split tiles itself), v and x steps, next pre-step
        KP_TRY(adjoint_to_grid(p, p->d_u, KP_C64, nullptr, st, /*splits_zeroed=*/false));
        KP_TRY(adjoint_primal(p, KP_REG_TV, lambda, st));
        KP_TRY(pre_only(p, p->d_xbar, st));
        k_advance<<<1, 1, 0, st>>>(p->d_iter);
        KP_LAUNCH_CHECK();
        p->launches += 1;
        mark(p, PH_OTHER, st);
        return KP_OK;
    }
    if (levels_primal(p)) {
        // the primal step as separate kernels over the whole GPU: combine + step (z, or x and
        // xbar for l2), the wavelet levels (the last inverse level extrapolates and writes the
        // next forward grid) or the pre-step, the counter
        KP_TRY(adjoint_to_grid(p, p->d_u, KP_C64, nullptr, st, /*splits_zeroed=*/false));
        KP_TRY(adjoint_primal(p, reg, lambda, st));
        if (reg == KP_REG_L1_WAVELET) KP_TRY(wavelet_prox_levels(p, lambda, st));
        else KP_TRY(pre_only(p, p->d_xbar, st));
        k_advance<<<1, 1, 0, st>>>(p->d_iter);
        KP_LAUNCH_CHECK();
        p->launches += 1;
        mark(p, PH_OTHER, st);
        return KP_OK;
    }
    KP_TRY(adjoint_to_grid(p, p->d_u, KP_C64, nullptr, st, /*splits_zeroed=*/true));
    if (reg == KP_REG_L1_WAVELET && cluster_prox_ok(p)) KP_TRY(primal_cluster(p, lambda, st));
    else KP_TRY(primal_fused(p, reg, lambda, st));
    mark(p, PH_OTHER, st);
    return KP_OK;
}

static void drop_graph(Graph& gr) {
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
    if (gr.graph) cudaGraphDestroy(gr.graph);
    gr.exec = nullptr;
    gr.graph = nullptr;
}

void drop_graphs(kp_plan p) {
    for (auto& gr : p->graphs) drop_graph(gr);
    p->graph_gen++;
}

// Capture one iteration on the plan's private stream; replay it on the caller's stream.
static kp_status get_graph(kp_plan p, int reg, float lambda, Graph** out) {
    Graph& gr = p->graphs[reg];
    const int key = (int)p->ys_t * 4 + reg;
    if (gr.exec && gr.reg == key && gr.lambda == lambda && gr.n_items == p->n_items) { *out = &gr; return KP_OK; }
    drop_graph(gr);
    cudaStream_t cs = p->cap_stream;
    const int64_t before = p->launches;
    KP_TRY_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    kp_status s = issue_iteration(p, reg, lambda, cs);
    gr.launches = p->launches - before;
    p->launches = before;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (s != KP_OK) { if (graph) cudaGraphDestroy(graph); return s; }
    KP_TRY_CUDA(e);
    gr.graph = graph;
    KP_TRY_CUDA(cudaGraphInstantiate(&gr.exec, graph, 0));
    gr.reg = key;
    gr.lambda = lambda;
    gr.n_items = p->n_items;
    *out = &gr;
    return KP_OK;
}

static kp_status objective(kp_plan p, int reg, float lambda, double* F, cudaStream_t st) {
    const Geom& g = p->geo;
    const int64_t CM = (int64_t)g.C * g.M;
    KP_TRY(forward_to(p, p->d_x, p->d_kt, KP_C64, nullptr, st));
    KP_TRY_CUDA(cudaMemsetAsync(p->d_red + 1, 0, 2 * sizeof(double), st));
    const unsigned b = (unsigned)std::min<int64_t>(nblk(CM, 256), 1216);
    switch (p->ys_t) {
        case KP_C64: k_resid2<float2><<<b, 256, 0, st>>>(p->d_kt, (const float2*)p->d_ys, CM, p->d_red + 1); break;
        case KP_C32_BF16: k_resid2<__nv_bfloat162><<<b, 256, 0, st>>>(p->d_kt, (const __nv_bfloat162*)p->d_ys, CM, p->d_red + 1); break;
        default: k_resid2<__half2><<<b, 256, 0, st>>>(p->d_kt, (const __half2*)p->d_ys, CM, p->d_red + 1); break;
    }
    KP_LAUNCH_CHECK();
    const unsigned bn = (unsigned)std::min<int64_t>(nblk(g.N, 256), 1216);
    if (reg == KP_REG_L2) {
        k_norm2<<<bn, 256, 0, st>>>(p->d_x, g.N, p->d_red + 2);
    } else if (reg == KP_REG_TV) {
        KP_TRY(tv_sumabs(p, p->d_x, p->d_red + 2, st));
    } else {
        KP_TRY(wavelet_apply(p, p->d_x, p->d_w, true, st));
        k_sumabs<<<bn, 256, 0, st>>>(p->d_w, g.N, p->d_red + 2);
    }
    KP_LAUNCH_CHECK();
    double h[2];
    KP_TRY_CUDA(cudaMemcpyAsync(h, p->d_red + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    KP_TRY_CUDA(cudaStreamSynchronize(st));
    *F = 0.5 * h[0] + (reg == KP_REG_L2 ? 0.5 * lambda * h[1] : lambda * h[1]);
    return KP_OK;
}

static kp_status ensure_sched(kp_plan p, int iters) {
    if (iters <= p->sched_cap) return KP_OK;
    if (p->d_sched) cudaFree(p->d_sched);
    p->d_sched = nullptr;
    const int cap = std::max(iters, 128);
    KP_TRY_CUDA(cudaMalloc(&p->d_sched, 3 * (size_t)cap * sizeof(float)));
    p->sched_cap = cap;
    drop_graphs(p);   // graphs bake the schedule pointer in
    return KP_OK;
}

// The TV dual variable v [D][N], allocated at the plan's first TV solve.
kp_status ensure_tv_dual(kp_plan p) {
    if (p->d_v) return KP_OK;
    KP_TRY_CUDA(cudaMalloc(&p->d_v, (size_t)p->geo.D * p->geo.N * sizeof(float2)));
    drop_graphs(p);
    return KP_OK;
}

// Everything a PDHG run needs before its first iteration (Sec. 4.1): measurements and
// preconditioner in sorted order, min p, lambda_max (given, or 30 power iterations), the
// step-size schedule, the initial iterates (zero, or a caller's state whose dual variable is
// brought into sorted order) and the forward grid of xbar.
// The measurements into sorted order (their first reader is the first dual step).
kp_status solve_measurements(kp_plan plan, const void* y_dev, kp_cdtype y_t, cudaStream_t st) {
    const Geom& g = plan->geo;
    plan->ys_t = y_t;
    if (y_t == KP_C64) k_permute<float2><<<nblk(g.M, 256), 256, 0, st>>>((const float2*)y_dev, (float2*)plan->d_ys, plan->d_perm, g.M, g.C);
    else k_permute<unsigned><<<nblk(g.M, 256), 256, 0, st>>>((const unsigned*)y_dev, (unsigned*)plan->d_ys, plan->d_perm, g.M, g.C);
    KP_LAUNCH_CHECK();
    plan->launches += 1;
    return KP_OK;
}

kp_status solve_setup_a(kp_plan plan, const void* y_dev, kp_cdtype y_t, const float* p_dev, int iters, cudaStream_t st,
                        const kp_pdhg_state* start) {
    const Geom& g = plan->geo;
    const int k0 = start ? start->k : 0;
    KP_TRY(ensure_sched(plan, std::max(iters + k0, 1)));
    plan->ys_t = y_t;
    if (y_dev) KP_TRY(solve_measurements(plan, y_dev, y_t, st));
    // preconditioner
    const float* pu = p_dev;
    if (!pu) {
        // no wait here: entries whose denominator was not positive are left at 0 and
        // reported through the min-p check below
        KP_TRY(make_preconditioner_enqueue(plan, 1, plan->d_puser, st));
        pu = plan->d_puser;
    }
    k_permute<float><<<nblk(g.M, 256), 256, 0, st>>>(pu, plan->d_ps, plan->d_perm, g.M, g.C);
    KP_LAUNCH_CHECK();
    KP_TRY_CUDA(cudaMemsetAsync(plan->d_flag, 0, KP_NFLAGS * sizeof(int), st));
    {
        static const int init = 0x7f7fffff;
        KP_TRY_CUDA(cudaMemcpyAsync(plan->d_flag + 4, &init, sizeof(int), cudaMemcpyHostToDevice, st));
        const int64_t CM = (int64_t)g.C * g.M;
        k_pmin<<<(unsigned)std::min<int64_t>(nblk(CM, 256), 1216), 256, 0, st>>>(plan->d_ps, CM, plan->d_flag + 4, plan->d_flag + 5);
        KP_LAUNCH_CHECK();
    }
    plan->launches += 2;
    return KP_OK;
}

kp_status solve_setup_b(kp_plan plan, int iters, cudaStream_t st, int reg, const kp_pdhg_state* start) {
    const Geom& g = plan->geo;
    const int k0 = start ? start->k : 0;
    iters += k0;                       // the schedule runs from iteration 0; the run starts at k0
    k_schedule<<<1, 1, 0, st>>>(plan->d_schedd, plan->d_flag + 4, std::max(iters, 1), plan->d_sched, plan->d_flag + 6,
                                reg == KP_REG_TV ? g.D : 0);
    KP_LAUNCH_CHECK();
    plan->launches += 1;
    if (!start) {
        // x0 = xbar0 = 0, u0 = 0
        KP_TRY_CUDA(cudaMemsetAsync(plan->d_x, 0, g.N * sizeof(float2), st));
        KP_TRY_CUDA(cudaMemsetAsync(plan->d_xbar, 0, g.N * sizeof(float2), st));
        KP_TRY_CUDA(cudaMemsetAsync(plan->d_u, 0, (size_t)g.C * g.M * sizeof(float2), st));
    } else {
        // a caller's state: x_k, xbar_k, u_k (user sample order -> sorted)
        KP_TRY_CUDA(cudaMemcpyAsync(plan->d_x, start->x, g.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        KP_TRY_CUDA(cudaMemcpyAsync(plan->d_xbar, start->xbar, g.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        k_permute<float2><<<nblk(g.M, 256), 256, 0, st>>>((const float2*)start->u, plan->d_u, plan->d_perm, g.M, g.C);
        KP_LAUNCH_CHECK();
        plan->launches += 1;
    }
    if (reg == KP_REG_TV) {
        KP_TRY(ensure_tv_dual(plan));
        if (start) KP_TRY_CUDA(cudaMemcpyAsync(plan->d_v, start->v, (size_t)g.D * g.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        else KP_TRY_CUDA(cudaMemsetAsync(plan->d_v, 0, (size_t)g.D * g.N * sizeof(float2), st));   // v_0 = 0
    }
    k_set_int<<<1, 1, 0, st>>>(plan->d_iter, k0);
    KP_LAUNCH_CHECK();
    plan->launches += 1;
    KP_TRY_CUDA(cudaMemsetAsync(plan->d_bar, 0, 4 * sizeof(unsigned int), st));   // grid-barrier counter
    // forward grid of xbar (the primal step writes the next one each iteration)
    if (!start) KP_TRY_CUDA(cudaMemsetAsync(plan->d_grid, 0, (size_t)g.C * g.G * sizeof(float2), st));
    else KP_TRY(pre_only(plan, plan->d_xbar, st));
    // split tiles of the spreading grid start at zero (the primal step re-clears them)
    KP_TRY(zero_split_only(plan, st));
    (void)cluster_prox_ok(plan);   // decide the primal path here, outside any graph capture
    return KP_OK;
}


// Everything a PDHG run needs before its first iteration (Sec. 4.1): measurements and
// preconditioner in sorted order, min p, lambda_max (given, or 30 power iterations), the
// step-size schedule, the initial iterates (zero, or a caller's state whose dual variable is
// brought into sorted order) and the forward grid of xbar.
kp_status solve_setup(kp_plan plan, const void* y_dev, kp_cdtype y_t, const float* p_dev, double lmax, int iters,
                      cudaStream_t st, int reg, const kp_pdhg_state* start, cudaEvent_t y_ready) {
    const Geom& g = plan->geo;
    // with y_ready (measurements still being copied in), they are loaded after the power method
    KP_TRY(solve_setup_a(plan, y_ready ? nullptr : y_dev, y_t, p_dev, iters, st, start));
    // lambda_max(P A A^H)
    if (lmax > 0) {
        k_set_double<<<1, 1, 0, st>>>(plan->d_schedd, lmax);
        KP_LAUNCH_CHECK();
        plan->launches += 1;
    } else {
        KP_TRY(fill_image(plan->d_z, g.N, make_float2(1.f, 0.f), st));
        plan->launches += 1;
        KP_TRY(power_method(plan, plan->d_ps, 30, st));
    }
    if (y_ready) {
        KP_TRY_CUDA(cudaStreamWaitEvent(st, y_ready, 0));
        KP_TRY(solve_measurements(plan, y_dev, y_t, st));
    }
    return solve_setup_b(plan, iters, st, reg, start);
}

kp_status pdhg_iteration(kp_plan p, int reg, float lambda, cudaStream_t st) { return issue_iteration(p, reg, lambda, st); }

// The same iteration without the cooperative primal kernel (for several plans running
// concurrently): adjoint + primal step kernel, wavelet level kernels (threshold, extrapolation
// and the next pre-step fused into them) or the pre-step kernel for l2, counter kernel.
kp_status pdhg_iteration_concurrent(kp_plan p, int reg, float lambda, cudaStream_t st) {
    KP_TRY(fft_forward_only(p, st));
    KP_TRY(interp_dual_only(p, st));
    KP_TRY(adjoint_to_grid(p, p->d_u, KP_C64, nullptr, st));
    KP_TRY(adjoint_primal(p, reg, lambda, st));   // TV: dual step on v, then the primal step
    if (reg == KP_REG_L1_WAVELET) KP_TRY(wavelet_prox_levels(p, lambda, st));
    else KP_TRY(pre_only(p, p->d_xbar, st));
    k_advance<<<1, 1, 0, st>>>(p->d_iter);
    KP_LAUNCH_CHECK();
    p->launches += 1;
    return KP_OK;
}

// ---------------------------------------------------------------- l2 through the dual
// (A A^H + lambda I) w = lambda y by conjugate gradients with the diagonal p as preconditioner
// (appendix on the connection to Trzasko et al.), in the plan's sorted sample order, with the
// scalars on the device so that no iteration waits for the host; x = A^H w / lambda.
// s[0] = <r, p r>, s[1] = <d, q>, s[2] = the next <r, p r>, s[3] = ||r||^2, s[4] = alpha,
// s[5] = beta.

// w = 0, r = lambda y, d = p r; s[0] += <r, p r>, s[3] += ||r||^2
__global__ void k_cg_init(const float2* __restrict__ ys, const float* __restrict__ ps, int64_t n, float lambda,
                          float2* __restrict__ w, float2* __restrict__ r, float2* __restrict__ d,
                          double* __restrict__ s) {
    double a = 0, b = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 y = ys[i];
        const float pi = ps ? ps[i] : 1.f;
        const float2 ri = make_float2(lambda * y.x, lambda * y.y);
        w[i] = make_float2(0.f, 0.f);
        r[i] = ri;
        d[i] = make_float2(pi * ri.x, pi * ri.y);
        const double m2 = (double)ri.x * ri.x + (double)ri.y * ri.y;
        a += pi * m2;
        b += m2;
    }
    block_sum_to<int>(a, s);
    __syncthreads();
    block_sum_to<int>(b, s + 3);
}

// q <- q + lambda d (q = A A^H d on entry); s[1] += Re <d, q>
__global__ void k_cg_dq(float2* __restrict__ q, const float2* __restrict__ d, int64_t n, float lambda,
                        double* __restrict__ s) {
    double a = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 di = d[i];
        float2 qi = q[i];
        qi.x += lambda * di.x;
        qi.y += lambda * di.y;
        q[i] = qi;
        a += (double)di.x * qi.x + (double)di.y * qi.y;
    }
    block_sum_to<int>(a, s + 1);
}

// mode 0: alpha = s[0] / s[1]; mode 1: beta = s[2] / s[0], trace[k] = ||r||, s[0] = s[2] and
// the accumulators cleared; mode 2 (start): trace[k] = ||r||, s[3] cleared.  A zero
// denominator (the residual vanished) gives a zero step.
__global__ void k_cg_scalars(double* __restrict__ s, int mode, double* __restrict__ trace, int k,
                             int* __restrict__ bad) {
    if (mode == 0) {
        s[4] = s[1] > 0 ? s[0] / s[1] : 0.0;
        return;
    }
    trace[k] = sqrt(s[3]);
    if (!isfinite(s[3])) *bad = 1;
    if (mode == 2) {
        s[3] = 0.0;
        return;
    }
    s[5] = s[0] > 0 ? s[2] / s[0] : 0.0;
    s[0] = s[2];
    s[1] = 0.0;
    s[2] = 0.0;
    s[3] = 0.0;
}

// w += alpha d, r -= alpha q; s[2] += <r, p r>, s[3] += ||r||^2
__global__ void k_cg_step(float2* __restrict__ w, float2* __restrict__ r, const float2* __restrict__ d,
                          const float2* __restrict__ q, const float* __restrict__ ps, int64_t n,
                          double* __restrict__ s) {
    const float alpha = (float)s[4];
    double a = 0, b = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 di = d[i], qi = q[i];
        float2 wi = w[i], ri = r[i];
        wi.x += alpha * di.x;
        wi.y += alpha * di.y;
        ri.x -= alpha * qi.x;
        ri.y -= alpha * qi.y;
        w[i] = wi;
        r[i] = ri;
        const double m2 = (double)ri.x * ri.x + (double)ri.y * ri.y;
        a += (ps ? ps[i] : 1.f) * m2;
        b += m2;
    }
    block_sum_to<int>(a, s + 2);
    __syncthreads();
    block_sum_to<int>(b, s + 3);
}

// d = p r + beta d
__global__ void k_cg_dir(float2* __restrict__ d, const float2* __restrict__ r, const float* __restrict__ ps, int64_t n,
                         const double* __restrict__ s) {
    const float beta = (float)s[5];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float pi = ps ? ps[i] : 1.f;
        const float2 ri = r[i], di = d[i];
        d[i] = make_float2(pi * ri.x + beta * di.x, pi * ri.y + beta * di.y);
    }
}

__global__ void k_scale_copy(const float2* __restrict__ in, float2* __restrict__ out, int64_t n, float a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2(a * in[i].x, a * in[i].y);
}

static kp_status dual_l2(kp_plan p, const float2* y_dev, const float* p_dev, float lambda, int iters, float2* x_dev,
                         double* res_trace, cudaStream_t st) {
    const Geom& g = p->geo;
    const int64_t n = (int64_t)g.C * g.M;
    if (n > p->cg_cap) {
        if (p->d_cg_r) cudaFree(p->d_cg_r);
        if (p->d_cg_d) cudaFree(p->d_cg_d);
        p->d_cg_r = p->d_cg_d = nullptr;
        p->cg_cap = 0;
        KP_TRY_CUDA(cudaMalloc(&p->d_cg_r, n * sizeof(float2)));
        KP_TRY_CUDA(cudaMalloc(&p->d_cg_d, n * sizeof(float2)));
        p->cg_cap = n;
    }
    if (iters + 1 > p->cg_trace_cap) {
        if (p->d_cg_trace) cudaFree(p->d_cg_trace);
        p->d_cg_trace = nullptr;
        p->cg_trace_cap = 0;
        KP_TRY_CUDA(cudaMalloc(&p->d_cg_trace, (size_t)(iters + 1) * sizeof(double)));
        p->cg_trace_cap = iters + 1;
    }
    // measurements and preconditioner into sorted order; min p and its sign check
    k_permute<float2><<<nblk(g.M, 256), 256, 0, st>>>(y_dev, (float2*)p->d_ys, p->d_perm, g.M, g.C);
    KP_LAUNCH_CHECK();
    const float* ps = nullptr;
    KP_TRY_CUDA(cudaMemsetAsync(p->d_flag, 0, KP_NFLAGS * sizeof(int), st));
    if (p_dev) {
        k_permute<float><<<nblk(g.M, 256), 256, 0, st>>>(p_dev, p->d_ps, p->d_perm, g.M, g.C);
        static const int init = 0x7f7fffff;
        KP_TRY_CUDA(cudaMemcpyAsync(p->d_flag + 4, &init, sizeof(int), cudaMemcpyHostToDevice, st));
        k_pmin<<<(unsigned)std::min<int64_t>(nblk(n, 256), 1216), 256, 0, st>>>(p->d_ps, n, p->d_flag + 4, p->d_flag + 5);
        KP_LAUNCH_CHECK();
        ps = p->d_ps;
        p->launches += 2;
    }
    p->launches += 1;
    float2* w = p->d_u;
    float2* r = p->d_cg_r;
    float2* d = p->d_cg_d;
    float2* q = p->d_kt;
    double* s = p->d_red + 8;     // 6 scalars (d_red holds 16)
    int* bad = p->d_flag + 6;
    const unsigned nb = (unsigned)std::min<int64_t>(nblk(n, 256), 1216);
    KP_TRY_CUDA(cudaMemsetAsync(s, 0, 6 * sizeof(double), st));
    k_cg_init<<<nb, 256, 0, st>>>((const float2*)p->d_ys, ps, n, lambda, w, r, d, s);
    k_cg_scalars<<<1, 1, 0, st>>>(s, 2, p->d_cg_trace, 0, bad);   // trace[0] = ||lambda y||
    KP_LAUNCH_CHECK();
    p->launches += 2;
    for (int k = 0; k < iters; ++k) {
        KP_TRY(adjoint_to_grid(p, d, KP_C64, nullptr, st));              // A^H d (sorted order in)
        KP_TRY(grid_to_image(p, p->d_w, st));
        KP_TRY(forward_to(p, p->d_w, q, KP_C64, nullptr, st));            // A A^H d (sorted order out)
        k_cg_dq<<<nb, 256, 0, st>>>(q, d, n, lambda, s);
        k_cg_scalars<<<1, 1, 0, st>>>(s, 0, p->d_cg_trace, k + 1, bad);
        k_cg_step<<<nb, 256, 0, st>>>(w, r, d, q, ps, n, s);
        k_cg_scalars<<<1, 1, 0, st>>>(s, 1, p->d_cg_trace, k + 1, bad);
        k_cg_dir<<<nb, 256, 0, st>>>(d, r, ps, n, s);
        KP_LAUNCH_CHECK();
        p->launches += 5;
    }
    // x = A^H w / lambda
    KP_TRY(adjoint_to_grid(p, w, KP_C64, nullptr, st));
    KP_TRY(grid_to_image(p, p->d_w, st));
    k_scale_copy<<<nblk(g.N, 256), 256, 0, st>>>(p->d_w, x_dev, g.N, 1.f / lambda);
    KP_LAUNCH_CHECK();
    p->launches += 1;
    int flags[KP_NFLAGS];
    KP_TRY_CUDA(cudaMemcpyAsync(flags, p->d_flag, KP_NFLAGS * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (res_trace)
        KP_TRY_CUDA(cudaMemcpyAsync(res_trace, p->d_cg_trace, (size_t)(iters + 1) * sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
    KP_TRY_CUDA(cudaStreamSynchronize(st));
    if (flags[5] != 0) { set_error(std::to_string(flags[5]) + " preconditioner entries are not positive and finite"); return KP_EINVAL; }
    if (flags[6] != 0) { set_error("a residual of the dual conjugate gradients is not finite"); return KP_ENONFINITE; }
    return KP_OK;
}

}  // namespace kp

using namespace kp;

extern "C" {

kp_status kp_dual_l2_solve(kp_plan plan, const void* y_dev, const float* p_dev, float lambda, int iters, void* x_dev,
                           double* res_trace, void* stream) {
    KP_RANGE("kp_dual_l2_solve");
    if (!plan || !y_dev || !x_dev) { set_error("null argument"); return KP_EINVAL; }
    if (!plan->traj_set || !plan->maps_set) { set_error("trajectory and maps must be set"); return KP_EINVAL; }
    if (iters < 0) { set_error("iters must be >= 0"); return KP_EINVAL; }
    if (!(lambda > 0.f) || !std::isfinite(lambda)) { set_error("lambda must be finite and > 0"); return KP_EINVAL; }
    return dual_l2(plan, (const float2*)y_dev, p_dev, lambda, iters, (float2*)x_dev, res_trace, (cudaStream_t)stream);
}

kp_status kp_wavelet(kp_plan plan, const void* in_dev, void* out_dev, int forward, void* stream) {
    KP_RANGE("kp_wavelet");
    if (!plan || !in_dev || !out_dev) { set_error("null argument"); return KP_EINVAL; }
    if (plan->P.wavelet_levels < 1) { set_error("plan has wavelet_levels = 0"); return KP_EINVAL; }
    return wavelet_apply(plan, (const float2*)in_dev, (float2*)out_dev, forward != 0, (cudaStream_t)stream);
}

kp_status kp_max_eig(kp_plan plan, const float* p_dev, const void* v0_dev, int iters, double* lmax, void* stream) {
    KP_RANGE("kp_max_eig");
    if (!plan || !lmax) { set_error("null argument"); return KP_EINVAL; }
    if (iters < 1) { set_error("iters must be >= 1"); return KP_EINVAL; }
    if (!plan->traj_set || !plan->maps_set) { set_error("trajectory and maps must be set"); return KP_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const Geom& g = plan->geo;
    if (p_dev) {
        k_permute<float><<<nblk(g.M, 256), 256, 0, st>>>(p_dev, plan->d_ps, plan->d_perm, g.M, g.C);
        KP_LAUNCH_CHECK();
        plan->launches += 1;
    }
    if (v0_dev) KP_TRY_CUDA(cudaMemcpyAsync(plan->d_z, v0_dev, g.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    else { KP_TRY(fill_image(plan->d_z, g.N, make_float2(1.f, 0.f), st)); plan->launches += 1; }
    KP_TRY(power_method(plan, p_dev ? plan->d_ps : nullptr, iters, st));
    KP_TRY_CUDA(cudaMemcpyAsync(lmax, plan->d_schedd, sizeof(double), cudaMemcpyDeviceToHost, st));
    KP_TRY_CUDA(cudaStreamSynchronize(st));
    if (!(*lmax > 0) || !std::isfinite(*lmax)) { set_error("power method norm is zero or not finite"); return KP_ENONFINITE; }
    return KP_OK;
}

static kp_status ensure_events(kp_plan p, int n) {
    if (n <= p->ev_cap) return KP_OK;
    for (int i = 0; i < p->ev_cap; ++i) cudaEventDestroy(p->ev[i]);
    delete[] p->ev;
    delete[] p->ev_phase;
    p->ev = new cudaEvent_t[n];
    p->ev_phase = new int[n];
    p->ev_cap = 0;
    for (int i = 0; i < n; ++i) {
        KP_TRY_CUDA(cudaEventCreate(&p->ev[i]));
        p->ev_cap = i + 1;
    }
    return KP_OK;
}

static kp_status pdhg_solve_impl(kp_plan plan, const void* y_dev, kp_cdtype y_t, const float* p_dev, kp_reg reg,
                                 float lambda, int iters, double lmax, const kp_pdhg_state* start, kp_pdhg_state* end,
                                 double* obj_trace, kp_stats* stats, void* stream, cudaEvent_t y_ready);

kp_status kp_pdhg_solve_ex(kp_plan plan, const void* y_dev, kp_cdtype y_t, const float* p_dev, kp_reg reg,
                           float lambda, int iters, double lmax, const kp_pdhg_state* start, kp_pdhg_state* end,
                           double* obj_trace, kp_stats* stats, void* stream) {
    KP_RANGE("kp_pdhg_solve_ex");
    return pdhg_solve_impl(plan, y_dev, y_t, p_dev, reg, lambda, iters, lmax, start, end, obj_trace, stats, stream,
                           nullptr);
}

static kp_status pdhg_solve_impl(kp_plan plan, const void* y_dev, kp_cdtype y_t, const float* p_dev, kp_reg reg,
                                 float lambda, int iters, double lmax, const kp_pdhg_state* start, kp_pdhg_state* end,
                                 double* obj_trace, kp_stats* stats, void* stream, cudaEvent_t y_ready) {
    if (!plan || !y_dev || !end || !end->x) { set_error("null argument"); return KP_EINVAL; }
    if (!plan->traj_set || !plan->maps_set) { set_error("trajectory and maps must be set"); return KP_EINVAL; }
    if (iters < 0) { set_error("iters must be >= 0"); return KP_EINVAL; }
    if (!(lambda >= 0.f) || !std::isfinite(lambda)) { set_error("lambda must be finite and >= 0"); return KP_EINVAL; }
    if (reg != KP_REG_L2 && reg != KP_REG_L1_WAVELET && reg != KP_REG_TV) { set_error("bad regulariser"); return KP_EINVAL; }
    if (reg == KP_REG_L1_WAVELET && plan->P.wavelet_levels < 1) { set_error("l1-wavelet needs wavelet_levels >= 1"); return KP_EINVAL; }
    if (y_t != KP_C64 && y_t != KP_C32_BF16 && y_t != KP_C32_FP16) { set_error("bad y type"); return KP_EINVAL; }
    if (start && (start->k < 0 || !start->x || !start->xbar || !start->u || (reg == KP_REG_TV && !start->v))) {
        set_error("a start state needs k >= 0 and x, xbar, u (and v for TV)");
        return KP_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const Geom& g = plan->geo;
    const int k0 = start ? start->k : 0;
    KP_TRY(solve_setup(plan, y_dev, y_t, p_dev, lmax, iters, st, (int)reg, start, y_ready));
    kp_status status = KP_OK;
    double F0 = 0, F = NAN;
    double phase_ms[PH_N] = {0};
    KP_PHASE("pdhg_iterations");
    if (iters > 0) {
        Graph* gr = nullptr;
        if (!plan->profiling) KP_TRY(get_graph(plan, (int)reg, lambda, &gr));
        else KP_TRY(ensure_events(plan, 16 * PH_N + 2));
        for (int k = 0; k < iters; ++k) {
            if (gr) {
                KP_TRY_CUDA(cudaGraphLaunch(gr->exec, st));
                plan->launches += gr->launches;
            } else {
                // profiled iteration: direct launches with an event at every phase boundary
                plan->ev_used = 0;
                KP_TRY(issue_iteration(plan, (int)reg, lambda, st));
                mark(plan, PH_N, st);
                KP_TRY_CUDA(cudaEventSynchronize(plan->ev[plan->ev_used - 1]));
                for (int e = 0; e + 1 < plan->ev_used; ++e) {
                    float ms = 0.f;
                    KP_TRY_CUDA(cudaEventElapsedTime(&ms, plan->ev[e], plan->ev[e + 1]));
                    phase_ms[plan->ev_phase[e]] += ms;
                }
                plan->ev_used = 0;
            }
            if (obj_trace) {
                KP_TRY(objective(plan, (int)reg, lambda, &F, st));
                KP_TRY(pre_only(plan, plan->d_xbar, st));   // the objective's forward reused d_grid
                obj_trace[k] = F;
                if (k == 0) F0 = F;
                if (!std::isfinite(F)) { status = KP_ENONFINITE; break; }
                if (k > 0 && F > 1e3 * F0 && F0 > 0) { status = KP_EDIVERGED; break; }
            }
        }
    }
    // the result, checked on the device, and the rest of the state
    k_nonfinite<<<(unsigned)std::min<int64_t>(nblk(g.N, 256), 1216), 256, 0, st>>>(plan->d_x, g.N,
                                                                                   plan->d_flag + KP_FLAG_NONFINITE);
    KP_LAUNCH_CHECK();
    plan->launches += 1;
    KP_TRY_CUDA(cudaMemcpyAsync(end->x, plan->d_x, g.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    if (end->xbar) KP_TRY_CUDA(cudaMemcpyAsync(end->xbar, plan->d_xbar, g.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    if (end->u) {
        k_unpermute_c64<<<nblk(g.M, 256), 256, 0, st>>>(plan->d_u, (float2*)end->u, plan->d_perm, g.M, g.C);
        KP_LAUNCH_CHECK();
        plan->launches += 1;
    }
    if (end->v && reg == KP_REG_TV)
        KP_TRY_CUDA(cudaMemcpyAsync(end->v, plan->d_v, (size_t)g.D * g.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    int flags[KP_NFLAGS];
    double sd[4];
    KP_TRY_CUDA(cudaMemcpyAsync(flags, plan->d_flag, KP_NFLAGS * sizeof(int), cudaMemcpyDeviceToHost, st));
    KP_TRY_CUDA(cudaMemcpyAsync(sd, plan->d_schedd, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    KP_TRY_CUDA(cudaStreamSynchronize(st));
    end->k = k0 + iters;
    if (stats) {
        stats->iters = iters;
        stats->lmax = sd[0];
        stats->pmin = sd[1];
        stats->sigma_last = sd[2];
        stats->tau_last = sd[3];
        stats->final_obj = obj_trace ? F : NAN;
        for (int i = 0; i < KP_NPHASES && i < PH_N; ++i) stats->phase_ms[i] = phase_ms[i];
    }
    if (flags[KP_FLAG_P_BAD] != 0) { set_error(std::to_string(flags[KP_FLAG_P_BAD]) + " preconditioner entries are not positive and finite"); return KP_EINVAL; }
    if (flags[KP_FLAG_SCHED_BAD] != 0) { set_error("lambda_max or min p is not positive and finite"); return KP_EINVAL; }
    if (flags[KP_FLAG_TIMEOUT] != 0)
        return report_timeout(plan, st, "a bounded device wait (bulk-copy staging of the interpolation or a grid barrier of "
                                        "the primal kernel) gave up");
    if (status == KP_OK && flags[KP_FLAG_NONFINITE] != 0) { set_error("the reconstruction holds a NaN or an Inf"); return KP_ENONFINITE; }
    if (status == KP_ENONFINITE) set_error("the objective is not finite");
    if (status == KP_EDIVERGED) set_error("the objective grew above 1e3 times its first value");
    return status;
}

kp_status kp_pdhg_solve(kp_plan plan, const void* y_dev, kp_cdtype y_t, const float* p_dev, kp_reg reg, float lambda,
                        int iters, double lmax, void* x_dev, double* obj_trace, kp_stats* stats, void* stream) {
    KP_RANGE("kp_pdhg_solve");
    if (!x_dev) { set_error("null argument"); return KP_EINVAL; }
    kp_pdhg_state end{x_dev, nullptr, nullptr, nullptr, 0};
    return kp_pdhg_solve_ex(plan, y_dev, y_t, p_dev, reg, lambda, iters, lmax, nullptr, &end, obj_trace, stats, stream);
}

kp_status kp_pdhg_solve_host(kp_plan plan, const void* y_host, kp_cdtype y_t, const float* p_dev, kp_reg reg,
                             float lambda, int iters, double lmax, void* x_dev, double* obj_trace, kp_stats* stats,
                             void* stream) {
    KP_RANGE("kp_pdhg_solve_host");
    if (!plan || !y_host || !x_dev) { set_error("null argument"); return KP_EINVAL; }
    if (y_t != KP_C64 && y_t != KP_C32_BF16 && y_t != KP_C32_FP16) { set_error("bad y type"); return KP_EINVAL; }
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, y_host) != cudaSuccess || at.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        set_error("y_host must be page-locked host memory");
        return KP_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)plan->geo.C * plan->geo.M * (y_t == KP_C64 ? sizeof(float2) : sizeof(unsigned));
    if (!plan->d_ystage || plan->ystage_bytes < bytes) {
        if (plan->d_ystage) {
            KP_TRY_CUDA(cudaStreamSynchronize(st));
            cudaFree(plan->d_ystage);
        }
        plan->d_ystage = nullptr;
        plan->ystage_bytes = 0;
        KP_TRY_CUDA(cudaMalloc(&plan->d_ystage, bytes));
        plan->ystage_bytes = bytes;
    }
    if (!plan->copy_stream) KP_TRY_CUDA(cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking));
    if (!plan->ev_copy_in) KP_TRY_CUDA(cudaEventCreateWithFlags(&plan->ev_copy_in, cudaEventDisableTiming));
    if (!plan->ev_copy_done) KP_TRY_CUDA(cudaEventCreateWithFlags(&plan->ev_copy_done, cudaEventDisableTiming));
    // the copy starts once earlier work on `stream` (which may still read the staging buffer) is done
    KP_TRY_CUDA(cudaEventRecord(plan->ev_copy_in, st));
    KP_TRY_CUDA(cudaStreamWaitEvent(plan->copy_stream, plan->ev_copy_in, 0));
    KP_TRY_CUDA(cudaMemcpyAsync(plan->d_ystage, y_host, bytes, cudaMemcpyHostToDevice, plan->copy_stream));
    KP_TRY_CUDA(cudaEventRecord(plan->ev_copy_done, plan->copy_stream));
    kp_pdhg_state end{};
    end.x = x_dev;
    return pdhg_solve_impl(plan, plan->d_ystage, y_t, p_dev, reg, lambda, iters, lmax, nullptr, &end, obj_trace, stats,
                           stream, plan->ev_copy_done);
}

}  // extern "C"
