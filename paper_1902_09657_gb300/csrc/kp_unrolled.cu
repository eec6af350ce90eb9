// Differentiation: trajectory gradients of the SENSE NUFFT pair and the unrolled l2 PDHG with
// a hand-written reverse sweep (the benchmark spec's differentiable configuration; the paper's
// method is Sec. 4.1 with g = lambda ||x||^2 / 2).
//
// Trajectory derivative (t = f g/n, taps fixed):
//   d y_c[i] / d f_{i,d} = (g_d/n_d) N^{-1/2} sum_taps phi'(t_d - k_d) prod_{e != d} phi(t_e - k_e) Xhat_c[k],
//   phi'(u) = I1(beta sqrt(s)) beta (-u) / (4 sqrt(s)), s = 1 - (u/2)^2  (width 4; -> -beta^2 u / 8 at s = 0).
// With complex gradients g = dL/dRe + i dL/dIm, a real loss gets
//   through y = A x:    dL/df_{i,d} = Re sum_c conj(g_c[i]) dy_c[i]/df_{i,d}
//   through x = A^H u:  dL/df_{i,d} = Re sum_c conj(u_c[i]) d(A g_x)_c[i]/df_{i,d}.
//
// Unrolled PDHG: the forward runs the solver's own iteration (x_0 = xbar_0 = 0, u_0 = 0) and
// keeps, per iteration, xbar_k, u_{k+1} and x_{k+1} (per-iteration checkpoints); the backward
// walks them in reverse:
//   gx' = gx + (1 + theta) gxb;  glam += Re<gx', -tau c x_{k+1}>;  gv = c gx';  gx <- -theta gxb + gv
//   gu' = gu - tau A gv;  gf += -tau dtraj(u_{k+1}, gv)
//   gu <- gu' / (1 + sigma p);  gr = sigma p gu' / (1 + sigma p);  gy -= gr;  gxb <- A^H gr;  gf += dtraj(gr, xbar_k)
// with c = 1/(1 + tau lambda); p, lambda_max and the step sizes are held constant.
#include "kp_internal.cuh"

#include <cmath>
#include <vector>

namespace kp {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ float kb_w(float u, float beta) {
    const float h = 0.5f * u;
    const float a = 1.f - h * h;
    return a >= 0.f ? cyl_bessel_i0f(beta * sqrtf(a)) : 0.f;
}

__device__ __forceinline__ float kb_dw(float u, float beta) {
    const float h = 0.5f * u;
    const float s = 1.f - h * h;
    if (s < 0.f) return 0.f;
    if (s < 1e-10f) return -beta * beta * u * 0.125f;
    const float rs = sqrtf(s);
    return cyl_bessel_i1f(beta * rs) * beta * (-u) / (4.f * rs);
}

__device__ __forceinline__ int wrapk(int k, int g) { return k < 0 ? k + g : (k >= g ? k - g : k); }

// out[perm[s]][d] (+)= coeff * (g_d/n_d) N^{-1/2} sum_c Re(conj(a_c) sum_taps dphi_d prod phi Xhat_c[k])
template <int D>
__global__ void k_traj_grad(const float* __restrict__ u0t, const int* __restrict__ k0t, const float2* __restrict__ grid,
                            const float2* __restrict__ a, const int* __restrict__ aperm, Geom geo,
                            const int* __restrict__ perm, float coeff, int accumulate, float* __restrict__ out) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= geo.M) return;
    float w[D][KW], dw[D][KW];
    int off[D][KW];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const float u0 = u0t[(int64_t)d * geo.M + s];      // t - ceil(t)
        const int k0 = k0t[(int64_t)d * geo.M + s];        // ceil(t) - W/2, wrapped
        int stride = 1;
        for (int e = d + 1; e < D; ++e) stride *= geo.g[e];
#pragma unroll
        for (int j = 0; j < KW; ++j) {
            const float u = u0 + (float)(KW / 2 - j);
            w[d][j] = kb_w(u, geo.beta[d]);
            dw[d][j] = kb_dw(u, geo.beta[d]);
            off[d][j] = wrapk(k0 + j, geo.g[d]) * stride;
        }
    }
    float acc[D];
#pragma unroll
    for (int d = 0; d < D; ++d) acc[d] = 0.f;
    const int64_t ai = aperm ? aperm[s] : s;
    constexpr int TAPS = D == 2 ? KW * KW : KW * KW * KW;
    for (int c = 0; c < geo.C; ++c) {
        const float2* base = grid + (size_t)c * geo.G;
        float2 S[D];
#pragma unroll
        for (int d = 0; d < D; ++d) S[d] = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < TAPS; ++q) {
            int j[D];
            int r = q;
#pragma unroll
            for (int d = D - 1; d >= 0; --d) { j[d] = r % KW; r /= KW; }
            int o = 0;
#pragma unroll
            for (int d = 0; d < D; ++d) o += off[d][j[d]];
            const float2 v = base[o];
#pragma unroll
            for (int d = 0; d < D; ++d) {
                float f = 1.f;
#pragma unroll
                for (int e = 0; e < D; ++e) f *= (e == d) ? dw[e][j[e]] : w[e][j[e]];
                S[d].x = fmaf(f, v.x, S[d].x);
                S[d].y = fmaf(f, v.y, S[d].y);
            }
        }
        const float2 av = a[(size_t)c * geo.M + ai];
#pragma unroll
        for (int d = 0; d < D; ++d) acc[d] += av.x * S[d].x + av.y * S[d].y;
    }
    const int64_t o = perm[s];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const float val = coeff * ((float)geo.g[d] / (float)geo.n[d]) * geo.rsqrtN * acc[d];
        float* dst = out + o * D + d;
        *dst = accumulate ? *dst + val : val;
    }
}

static kp_status traj_grad(kp_plan p, const float2* a, const int* aperm, float coeff, bool accumulate, float* out,
                           cudaStream_t st) {
    const Geom& g = p->geo;
    if (g.D == 2) k_traj_grad<2><<<nblk(g.M, 128), 128, 0, st>>>(p->d_t, p->d_k0, p->d_gridF, a, aperm, g, p->d_perm, coeff, accumulate, out);
    else k_traj_grad<3><<<nblk(g.M, 128), 128, 0, st>>>(p->d_t, p->d_k0, p->d_gridF, a, aperm, g, p->d_perm, coeff, accumulate, out);
    KP_LAUNCH_CHECK();
    p->launches += 1;
    return KP_OK;
}

// ---------------------------------------------------------------- reverse-sweep kernels
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// image part of the reverse step k (see the header comment); glam accumulates in *glam.
__global__ void k_bw_image(float2* __restrict__ gx, const float2* __restrict__ gxb, const float2* __restrict__ xnew,
                           float2* __restrict__ gv, int64_t N, const float* __restrict__ sched, int k, float lambda,
                           double* __restrict__ glam) {
    const float tau = sched[3 * k + 1], theta = sched[3 * k + 2];
    const float c = 1.f / (1.f + tau * lambda);
    double part = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = gx[i], b = gxb[i], xn = xnew[i];
        const float2 gn = make_float2(a.x + (1.f + theta) * b.x, a.y + (1.f + theta) * b.y);
        part += -(double)tau * c * ((double)gn.x * xn.x + (double)gn.y * xn.y);
        const float2 v = make_float2(c * gn.x, c * gn.y);
        gv[i] = v;
        gx[i] = make_float2(v.x - theta * b.x, v.y - theta * b.y);
    }
    __shared__ double ws[32];
    part = warp_sum_d(part);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = part;
    __syncthreads();
    if (w == 0) {
        part = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
        part = warp_sum_d(part);
        if (lane == 0) atomicAdd(glam, part);
    }
}

// k-space part: gu' = gu - tau A gv (A gv in agv), gu = gu'/(1 + sigma p), gr = sigma p gu'/(1 + sigma p), gy -= gr
__global__ void k_bw_kspace(float2* __restrict__ gu, float2* __restrict__ gr, float2* __restrict__ gy,
                            const float2* __restrict__ agv, const float* __restrict__ ps, int64_t CM,
                            const float* __restrict__ sched, int k) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= CM) return;
    const float sig = sched[3 * k], tau = sched[3 * k + 1];
    const float sp = sig * ps[i];
    const float inv = 1.f / (1.f + sp);
    const float2 a = gu[i], b = agv[i];
    const float2 gn = make_float2(a.x - tau * b.x, a.y - tau * b.y);
    gu[i] = make_float2(gn.x * inv, gn.y * inv);
    const float2 r = make_float2(sp * inv * gn.x, sp * inv * gn.y);
    gr[i] = r;
    const float2 yv = gy[i];
    gy[i] = make_float2(yv.x - r.x, yv.y - r.y);
}

__global__ void k_unpermute(const float2* __restrict__ in, float2* __restrict__ out, const int* __restrict__ perm,
                            int64_t M, int C) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const int64_t o = perm[s];
    for (int c = 0; c < C; ++c) out[(size_t)c * M + o] = in[(size_t)c * M + s];
}

static kp_status ensure_tape(kp_plan p, int iters) {
    const Geom& g = p->geo;
    const size_t per = 2 * (size_t)g.N + (size_t)g.C * g.M;
    const size_t need = per * (size_t)iters;
    if (need > p->tape_cap) {
        if (p->d_tape) cudaFree(p->d_tape);
        p->d_tape = nullptr;
        KP_TRY_CUDA(cudaMalloc(&p->d_tape, need * sizeof(float2)));
        p->tape_cap = need;
    }
    if (!p->d_bk) KP_TRY_CUDA(cudaMalloc(&p->d_bk, 2 * (size_t)g.C * g.M * sizeof(float2)));
    return KP_OK;
}

}  // namespace kp

using namespace kp;

extern "C" {

kp_status kp_sense_forward_traj_grad(kp_plan plan, const void* x_dev, const void* gy_dev, float* gtraj_dev, void* stream) {
    KP_RANGE("kp_sense_forward_traj_grad");
    if (!plan || !x_dev || !gy_dev || !gtraj_dev) { set_error("null argument"); return KP_EINVAL; }
    if (!plan->traj_set || !plan->maps_set) { set_error("trajectory and maps must be set"); return KP_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    KP_TRY(forward_grid_only(plan, (const float2*)x_dev, st));
    return traj_grad(plan, (const float2*)gy_dev, plan->d_perm, 1.f, false, gtraj_dev, st);
}

kp_status kp_sense_adjoint_traj_grad(kp_plan plan, const void* u_dev, const void* gx_dev, float* gtraj_dev, void* stream) {
    KP_RANGE("kp_sense_adjoint_traj_grad");
    if (!plan || !u_dev || !gx_dev || !gtraj_dev) { set_error("null argument"); return KP_EINVAL; }
    if (!plan->traj_set || !plan->maps_set) { set_error("trajectory and maps must be set"); return KP_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    KP_TRY(forward_grid_only(plan, (const float2*)gx_dev, st));
    return traj_grad(plan, (const float2*)u_dev, plan->d_perm, 1.f, false, gtraj_dev, st);
}

kp_status kp_unrolled_forward(kp_plan plan, const void* y_dev, const float* p_dev, float lambda, int iters, double lmax,
                              void* x_dev, void* stream) {
    KP_RANGE("kp_unrolled_forward");
    if (!plan || !y_dev || !x_dev) { set_error("null argument"); return KP_EINVAL; }
    if (!plan->traj_set || !plan->maps_set) { set_error("trajectory and maps must be set"); return KP_EINVAL; }
    if (iters < 1) { set_error("iters must be >= 1"); return KP_EINVAL; }
    if (!(lambda >= 0.f) || !std::isfinite(lambda)) { set_error("lambda must be finite and >= 0"); return KP_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const Geom& g = plan->geo;
    KP_TRY(solve_setup(plan, y_dev, KP_C64, p_dev, lmax, iters, st));
    KP_TRY(ensure_tape(plan, iters));
    const size_t per = 2 * (size_t)g.N + (size_t)g.C * g.M;
    for (int k = 0; k < iters; ++k) {
        float2* tk = plan->d_tape + per * k;
        KP_TRY_CUDA(cudaMemcpyAsync(tk, plan->d_xbar, g.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        KP_TRY(pdhg_iteration(plan, KP_REG_L2, lambda, st));
        KP_TRY_CUDA(cudaMemcpyAsync(tk + g.N, plan->d_u, (size_t)g.C * g.M * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        KP_TRY_CUDA(cudaMemcpyAsync(tk + g.N + (size_t)g.C * g.M, plan->d_x, g.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    }
    KP_TRY_CUDA(cudaMemcpyAsync(x_dev, plan->d_x, g.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    int flags[8];
    KP_TRY_CUDA(cudaMemcpyAsync(flags, plan->d_flag, 8 * sizeof(int), cudaMemcpyDeviceToHost, st));
    KP_TRY_CUDA(cudaStreamSynchronize(st));
    if (flags[5] != 0 || flags[6] != 0) { set_error("preconditioner or lambda_max not positive and finite"); return KP_EINVAL; }
    if (flags[KP_FLAG_TIMEOUT] != 0)
        return report_timeout(plan, st, "a bounded device wait (bulk-copy staging of the interpolation) gave up");
    plan->tape_iters = iters;
    plan->tape_lambda = lambda;
    return KP_OK;
}

kp_status kp_unrolled_backward(kp_plan plan, const void* gx_dev, void* gy_dev, double* glambda, float* gtraj_dev,
                               void* stream) {
    KP_RANGE("kp_unrolled_backward");
    if (!plan || !gx_dev) { set_error("null argument"); return KP_EINVAL; }
    if (plan->tape_iters < 1) { set_error("kp_unrolled_forward must run first"); return KP_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const Geom& g = plan->geo;
    const int K = plan->tape_iters;
    const float lambda = plan->tape_lambda;
    const int64_t CM = (int64_t)g.C * g.M;
    const size_t per = 2 * (size_t)g.N + (size_t)CM;
    float2* gx = plan->d_x;
    float2* gxb = plan->d_xbar;
    float2* gv = plan->d_z;
    float2* gu = plan->d_u;
    float2* gr = plan->d_bk;
    float2* gy = plan->d_bk + CM;
    double* glam = plan->d_red + 4;
    KP_TRY_CUDA(cudaMemcpyAsync(gx, gx_dev, g.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    KP_TRY_CUDA(cudaMemsetAsync(gxb, 0, g.N * sizeof(float2), st));
    KP_TRY_CUDA(cudaMemsetAsync(gu, 0, CM * sizeof(float2), st));
    KP_TRY_CUDA(cudaMemsetAsync(gy, 0, CM * sizeof(float2), st));
    KP_TRY_CUDA(cudaMemsetAsync(glam, 0, sizeof(double), st));
    if (gtraj_dev) KP_TRY_CUDA(cudaMemsetAsync(gtraj_dev, 0, (size_t)g.M * g.D * sizeof(float), st));
    std::vector<float> sched(3 * (size_t)K);
    KP_TRY_CUDA(cudaMemcpyAsync(sched.data(), plan->d_sched, 3 * (size_t)K * sizeof(float), cudaMemcpyDeviceToHost, st));
    KP_TRY_CUDA(cudaStreamSynchronize(st));
    const unsigned bn = (unsigned)std::min<int64_t>(nblk(g.N, 256), 1216);
    for (int k = K - 1; k >= 0; --k) {
        const float2* tk = plan->d_tape + per * k;
        const float2* xbar_k = tk;
        const float2* u_k1 = tk + g.N;
        const float2* x_k1 = tk + g.N + CM;
        const float tau = sched[3 * (size_t)k + 1];
        k_bw_image<<<bn, 256, 0, st>>>(gx, gxb, x_k1, gv, g.N, plan->d_sched, k, lambda, glam);
        KP_LAUNCH_CHECK();
        KP_TRY(forward_to(plan, gv, plan->d_kt, KP_C64, nullptr, st));        // A gv (sorted); d_gridF = spectrum of gv
        if (gtraj_dev) KP_TRY(traj_grad(plan, u_k1, nullptr, -tau, true, gtraj_dev, st));
        k_bw_kspace<<<nblk(CM, 256), 256, 0, st>>>(gu, gr, gy, plan->d_kt, plan->d_ps, CM, plan->d_sched, k);
        KP_LAUNCH_CHECK();
        KP_TRY(adjoint_to_grid(plan, gr, KP_C64, nullptr, st));
        KP_TRY(grid_to_image(plan, gxb, st));
        if (gtraj_dev) {
            KP_TRY(forward_grid_only(plan, xbar_k, st));
            KP_TRY(traj_grad(plan, gr, nullptr, 1.f, true, gtraj_dev, st));
        }
        plan->launches += 2;
    }
    if (gy_dev) {
        k_unpermute<<<nblk(g.M, 256), 256, 0, st>>>(gy, (float2*)gy_dev, plan->d_perm, g.M, g.C);
        KP_LAUNCH_CHECK();
        plan->launches += 1;
    }
    double gl = 0.0;
    KP_TRY_CUDA(cudaMemcpyAsync(&gl, glam, sizeof(double), cudaMemcpyDeviceToHost, st));
    KP_TRY_CUDA(cudaStreamSynchronize(st));
    if (glambda) *glambda = gl;
    return KP_OK;
}

}  // extern "C"
