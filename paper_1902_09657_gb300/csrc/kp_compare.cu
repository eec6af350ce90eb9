// Comparison solvers of Sec. 6 on the plan's SENSE NUFFT pair:
//   * conjugate gradients on (A^H A + lambda I) x = A^H y for the l2 problem, plain or
//     preconditioned by M = P + lambda I with P the l2-optimised circulant of App. B
//     (M^{-1} v = IDFT(DFT(v) / (eig(P) + lambda)));
//   * FISTA (Beck & Teboulle) on 1/2 ||A x - y||^2 + g(x), g = lambda ||x||^2 / 2 or
//     lambda ||W x||_1, step 1/L:
//       x_{k+1} = prox_{g/L}(z_k - A^H (A z_k - y) / L),  t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,
//       z_{k+1} = x_{k+1} + (t_k - 1)/t_{k+1} (x_{k+1} - x_k),  x_0 = z_0 = 0, t_0 = 1.
// Both record the objective F(x_k) of Eq. obj after every iteration, reduced in float64 on the
// device (CG keeps A x_k by the recurrence A x_{k+1} = A x_k + alpha A d_k, so the trace costs
// no extra NUFFT; FISTA applies A to x_{k+1} when a trace is requested).  k-space vectors live in
// the plan's sorted sample order.
#include "kp_internal.cuh"

#include <cmath>
#include <vector>

namespace kp {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
static inline unsigned rblk(int64_t n) { return (unsigned)std::min<int64_t>(nblk(n, 256), 1216); }

__device__ __forceinline__ void block_add(double v, double* out) {
    __shared__ double ws[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(out, v);
    }
    __syncthreads();
}

// Scalars of CG: s[0] <r, z>, s[1] <d, q>, s[2] next <r, z>, s[3] alpha, s[4] beta,
// s[5] ||A x - y||^2, s[6] ||x||^2.

// q <- q + lambda d; s[1] += Re <d, q>
__global__ void k_cg_q(float2* __restrict__ q, const float2* __restrict__ d, int64_t n, float lambda, double* s) {
    double a = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 di = d[i];
        float2 qi = q[i];
        qi.x = fmaf(lambda, di.x, qi.x);
        qi.y = fmaf(lambda, di.y, qi.y);
        q[i] = qi;
        a += (double)di.x * qi.x + (double)di.y * qi.y;
    }
    block_add(a, s + 1);
}

__global__ void k_cg_alpha(double* s) { s[3] = s[1] > 0 ? s[0] / s[1] : 0.0; }

// x += alpha d, r -= alpha q; s[6] += ||x||^2
__global__ void k_cg_xr(float2* __restrict__ x, float2* __restrict__ r, const float2* __restrict__ d,
                        const float2* __restrict__ q, int64_t n, double* s) {
    const float al = (float)s[3];
    double a = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float2 xi = x[i], ri = r[i];
        const float2 di = d[i], qi = q[i];
        xi.x = fmaf(al, di.x, xi.x);
        xi.y = fmaf(al, di.y, xi.y);
        ri.x = fmaf(-al, qi.x, ri.x);
        ri.y = fmaf(-al, qi.y, ri.y);
        x[i] = xi;
        r[i] = ri;
        a += (double)xi.x * xi.x + (double)xi.y * xi.y;
    }
    block_add(a, s + 6);
}

// ax += alpha ad (k-space); s[5] += ||ax - y||^2
__global__ void k_cg_ax(float2* __restrict__ ax, const float2* __restrict__ ad, const float2* __restrict__ y,
                        int64_t n, double* s) {
    const float al = (float)s[3];
    double a = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float2 v = ax[i];
        const float2 w = ad[i], yi = y[i];
        v.x = fmaf(al, w.x, v.x);
        v.y = fmaf(al, w.y, v.y);
        ax[i] = v;
        const double ex = (double)v.x - yi.x, ey = (double)v.y - yi.y;
        a += ex * ex + ey * ey;
    }
    block_add(a, s + 5);
}

// out[slot] += Re <a, b>
__global__ void k_dot_re(const float2* __restrict__ a, const float2* __restrict__ b, int64_t n, double* out) {
    double v = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 x = a[i], y = b[i];
        v += (double)x.x * y.x + (double)x.y * y.y;
    }
    block_add(v, out);
}

// beta = s[2] / s[0], s[0] = s[2]; trace[k] = 1/2 s[5] + lambda/2 s[6]; accumulators cleared
__global__ void k_cg_next(double* s, double lambda, double* trace, int k) {
    s[4] = s[0] > 0 ? s[2] / s[0] : 0.0;
    s[0] = s[2];
    trace[k] = 0.5 * s[5] + 0.5 * lambda * s[6];
    s[1] = s[2] = s[5] = s[6] = 0.0;
}

// d = z + beta d
__global__ void k_cg_dir(float2* __restrict__ d, const float2* __restrict__ z, int64_t n, const double* s) {
    const float b = (float)s[4];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 zi = z[i], di = d[i];
        d[i] = make_float2(fmaf(b, di.x, zi.x), fmaf(b, di.y, zi.y));
    }
}

// v *= 1 / (N (eig + lambda)) (between the forward and the unnormalised inverse DFT)
__global__ void k_circ_apply(float2* __restrict__ v, const float* __restrict__ eig, int64_t n, float lambda) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float sc = 1.f / ((float)n * (eig[i] + lambda));
    const float2 a = v[i];
    v[i] = make_float2(a.x * sc, a.y * sc);
}

__global__ void k_copy2(const float2* __restrict__ a, float2* __restrict__ b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

// ---- FISTA
// r <- r - y (r = A z on entry), k-space
__global__ void k_sub(float2* __restrict__ r, const float2* __restrict__ y, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 a = r[i], b = y[i];
    r[i] = make_float2(a.x - b.x, a.y - b.y);
}

// v = z - g / L; l2 prox folded in when shrink > 0: v /= (1 + lambda / L)
__global__ void k_fista_grad(const float2* __restrict__ z, const float2* __restrict__ g, int64_t n, float invL,
                             float shrink, float2* __restrict__ v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 a = z[i], b = g[i];
    v[i] = make_float2((a.x - invL * b.x) * shrink, (a.y - invL * b.y) * shrink);
}

// complex soft threshold S_t(c) = c max(0, 1 - t/|c|)
__global__ void k_soft(float2* __restrict__ c, int64_t n, float t) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 a = c[i];
    const float m = sqrtf(a.x * a.x + a.y * a.y);
    const float sc = m > t ? 1.f - t / m : 0.f;
    c[i] = make_float2(a.x * sc, a.y * sc);
}

// z = xn + mom (xn - x); x = xn
__global__ void k_fista_mom(float2* __restrict__ x, const float2* __restrict__ xn, float2* __restrict__ z, int64_t n,
                            float mom) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 a = xn[i], b = x[i];
    z[i] = make_float2(a.x + mom * (a.x - b.x), a.y + mom * (a.y - b.y));
    x[i] = a;
}

// out += sum |a - y|^2 (k-space residual)
__global__ void k_resid_sq(const float2* __restrict__ a, const float2* __restrict__ y, int64_t n, double* out) {
    double v = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 p = a[i], q = y[i];
        const double ex = (double)p.x - q.x, ey = (double)p.y - q.y;
        v += ex * ex + ey * ey;
    }
    block_add(v, out);
}

__global__ void k_sum_abs(const float2* __restrict__ a, int64_t n, double* out) {
    double v = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 p = a[i];
        v += sqrt((double)p.x * p.x + (double)p.y * p.y);
    }
    block_add(v, out);
}

// trace[k] = 1/2 s[0] + weight s[1]; s cleared
__global__ void k_obj_store(double* s, double weight, double* trace, int k) {
    trace[k] = 0.5 * s[0] + weight * s[1];
    s[0] = s[1] = 0.0;
}

__global__ void k_permute_c64(const float2* __restrict__ in, float2* __restrict__ out, const int* __restrict__ perm,
                              int64_t M, int C) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const int64_t o = perm[s];
    for (int c = 0; c < C; ++c) out[(size_t)c * M + s] = in[(size_t)c * M + o];
}

void compare_destroy(kp_plan p) {
    if (p->fft_img_ok) cufftDestroy(p->fft_img);
    p->fft_img_ok = false;
    void* bufs[] = {p->d_circ_eig, p->d_circ, p->d_cmp, p->d_cmp_s, p->d_cmp_trace};
    for (void* b : bufs)
        if (b) cudaFree(b);
    p->d_circ_eig = nullptr;
    p->d_circ = nullptr;
    p->d_cmp = nullptr;
    p->d_cmp_s = nullptr;
    p->d_cmp_trace = nullptr;
}

static kp_status cmp_buffers(kp_plan p, int iters) {
    const Geom& g = p->geo;
    if (!p->d_cmp) KP_TRY_CUDA(cudaMalloc(&p->d_cmp, 2 * (size_t)g.N * sizeof(float2)));
    if (!p->d_cmp_s) KP_TRY_CUDA(cudaMalloc(&p->d_cmp_s, 16 * sizeof(double)));
    if (iters > p->cmp_trace_cap) {
        if (p->d_cmp_trace) cudaFree(p->d_cmp_trace);
        p->d_cmp_trace = nullptr;
        p->cmp_trace_cap = 0;
        KP_TRY_CUDA(cudaMalloc(&p->d_cmp_trace, (size_t)std::max(iters, 1) * sizeof(double)));
        p->cmp_trace_cap = std::max(iters, 1);
    }
    return KP_OK;
}

// A^H of a sorted k-space vector into an image
static kp_status adjoint_sorted(kp_plan p, const float2* u, float2* x, cudaStream_t st) {
    KP_TRY(adjoint_to_grid(p, u, KP_C64, nullptr, st));
    return grid_to_image(p, x, st);
}

static kp_status cg_l2(kp_plan p, const float2* y_dev, float lambda, int iters, bool circ, float2* x_dev,
                       double* obj_trace, cudaStream_t st) {
    const Geom& g = p->geo;
    const int64_t N = g.N, CM = (int64_t)g.C * g.M;
    KP_TRY(cmp_buffers(p, iters));
    if (circ) {
        if (!p->circ_ok || p->circ_version != p->traj_version) KP_TRY(circulant_enqueue(p, st));
        KP_TRY_CUFFT(cufftSetStream(p->fft_img, st));
    }
    float2* x = p->d_x;
    float2* r = p->d_xbar;
    float2* z = circ ? p->d_z : r;            // no preconditioner: z = r
    float2* q = p->d_w;
    float2* d = p->d_cmp;
    float2* ys = (float2*)p->d_ys;
    float2* ax = p->d_u;
    float2* ad = p->d_kt;
    double* s = p->d_cmp_s;
    k_permute_c64<<<nblk(g.M, 256), 256, 0, st>>>(y_dev, ys, p->d_perm, g.M, g.C);
    KP_LAUNCH_CHECK();
    p->ys_t = KP_C64;
    KP_TRY_CUDA(cudaMemsetAsync(s, 0, 16 * sizeof(double), st));
    KP_TRY_CUDA(cudaMemsetAsync(x, 0, N * sizeof(float2), st));
    KP_TRY_CUDA(cudaMemsetAsync(ax, 0, CM * sizeof(float2), st));
    KP_TRY(adjoint_sorted(p, ys, r, st));     // r = b = A^H y
    const auto precond = [&]() -> kp_status {
        if (!circ) return KP_OK;
        KP_TRY_CUFFT(cufftExecC2C(p->fft_img, (cufftComplex*)r, (cufftComplex*)z, CUFFT_FORWARD));
        k_circ_apply<<<nblk(N, 256), 256, 0, st>>>(z, p->d_circ_eig, N, lambda);
        KP_LAUNCH_CHECK();
        KP_TRY_CUFFT(cufftExecC2C(p->fft_img, (cufftComplex*)z, (cufftComplex*)z, CUFFT_INVERSE));
        p->launches += 1;
        return KP_OK;
    };
    KP_TRY(precond());
    k_copy2<<<nblk(N, 256), 256, 0, st>>>(z, d, N);
    k_dot_re<<<rblk(N), 256, 0, st>>>(r, z, N, s + 0);
    KP_LAUNCH_CHECK();
    p->launches += 3;
    for (int k = 0; k < iters; ++k) {
        KP_TRY(forward_to(p, d, ad, KP_C64, nullptr, st));       // A d (sorted)
        KP_TRY(adjoint_sorted(p, ad, q, st));                     // A^H A d
        k_cg_q<<<rblk(N), 256, 0, st>>>(q, d, N, lambda, s);
        k_cg_alpha<<<1, 1, 0, st>>>(s);
        k_cg_xr<<<rblk(N), 256, 0, st>>>(x, r, d, q, N, s);
        k_cg_ax<<<rblk(CM), 256, 0, st>>>(ax, ad, ys, CM, s);
        KP_LAUNCH_CHECK();
        KP_TRY(precond());
        k_dot_re<<<rblk(N), 256, 0, st>>>(r, z, N, s + 2);
        k_cg_next<<<1, 1, 0, st>>>(s, (double)lambda, p->d_cmp_trace, k);
        k_cg_dir<<<rblk(N), 256, 0, st>>>(d, z, N, s);
        KP_LAUNCH_CHECK();
        p->launches += 8;
    }
    KP_TRY_CUDA(cudaMemcpyAsync(x_dev, x, N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    if (obj_trace && iters > 0)
        KP_TRY_CUDA(cudaMemcpyAsync(obj_trace, p->d_cmp_trace, iters * sizeof(double), cudaMemcpyDeviceToHost, st));
    int flag = 0;
    KP_TRY_CUDA(cudaMemcpyAsync(&flag, p->d_flag + KP_FLAG_TIMEOUT, sizeof(int), cudaMemcpyDeviceToHost, st));
    KP_TRY_CUDA(cudaStreamSynchronize(st));
    if (flag) return report_timeout(p, st, "a bounded device wait (bulk-copy staging of the interpolation) gave up");
    if (obj_trace)
        for (int k = 0; k < iters; ++k)
            if (!std::isfinite(obj_trace[k])) { set_error("the objective is not finite"); return KP_ENONFINITE; }
    return KP_OK;
}

static kp_status fista(kp_plan p, const float2* y_dev, int reg, float lambda, int iters, double L, float2* x_dev,
                       double* obj_trace, cudaStream_t st) {
    const Geom& g = p->geo;
    const int64_t N = g.N, CM = (int64_t)g.C * g.M;
    KP_TRY(cmp_buffers(p, iters));
    float2* x = p->d_x;
    float2* z = p->d_z;
    float2* v = p->d_xbar;
    float2* w = p->d_w;                  // gradient / wavelet coefficients
    float2* xn = p->d_cmp;
    float2* xt = p->d_cmp + N;           // wavelet coefficients of x for the objective
    float2* ys = (float2*)p->d_ys;
    float2* rk = p->d_kt;
    double* s = p->d_cmp_s;
    k_permute_c64<<<nblk(g.M, 256), 256, 0, st>>>(y_dev, ys, p->d_perm, g.M, g.C);
    KP_LAUNCH_CHECK();
    p->ys_t = KP_C64;
    KP_TRY_CUDA(cudaMemsetAsync(s, 0, 16 * sizeof(double), st));
    KP_TRY_CUDA(cudaMemsetAsync(x, 0, N * sizeof(float2), st));
    KP_TRY_CUDA(cudaMemsetAsync(z, 0, N * sizeof(float2), st));
    const float invL = (float)(1.0 / L);
    const float shrink = reg == KP_REG_L2 ? (float)(1.0 / (1.0 + lambda / L)) : 1.f;
    double t = 1.0;
    for (int k = 0; k < iters; ++k) {
        KP_TRY(forward_to(p, z, rk, KP_C64, nullptr, st));       // A z
        k_sub<<<nblk(CM, 256), 256, 0, st>>>(rk, ys, CM);
        KP_LAUNCH_CHECK();
        KP_TRY(adjoint_sorted(p, rk, w, st));                     // A^H (A z - y)
        k_fista_grad<<<nblk(N, 256), 256, 0, st>>>(z, w, N, invL, shrink, reg == KP_REG_L2 ? xn : v);
        KP_LAUNCH_CHECK();
        p->launches += 2;
        if (reg == KP_REG_L1_WAVELET) {
            KP_TRY(wavelet_apply(p, v, w, true, st));
            k_soft<<<nblk(N, 256), 256, 0, st>>>(w, N, (float)(lambda / L));
            KP_LAUNCH_CHECK();
            KP_TRY(wavelet_apply(p, w, xn, false, st));
            p->launches += 1;
        }
        const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        k_fista_mom<<<nblk(N, 256), 256, 0, st>>>(x, xn, z, N, (float)((t - 1.0) / tn));
        KP_LAUNCH_CHECK();
        p->launches += 1;
        t = tn;
        if (obj_trace) {
            KP_TRY(forward_to(p, x, rk, KP_C64, nullptr, st));
            k_resid_sq<<<rblk(CM), 256, 0, st>>>(rk, ys, CM, s + 0);
            if (reg == KP_REG_L2) {
                k_dot_re<<<rblk(N), 256, 0, st>>>(x, x, N, s + 1);
            } else {
                KP_TRY(wavelet_apply(p, x, xt, true, st));
                k_sum_abs<<<rblk(N), 256, 0, st>>>(xt, N, s + 1);
            }
            k_obj_store<<<1, 1, 0, st>>>(s, reg == KP_REG_L2 ? 0.5 * lambda : (double)lambda, p->d_cmp_trace, k);
            KP_LAUNCH_CHECK();
            p->launches += 3;
        }
    }
    KP_TRY_CUDA(cudaMemcpyAsync(x_dev, x, N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    if (obj_trace && iters > 0)
        KP_TRY_CUDA(cudaMemcpyAsync(obj_trace, p->d_cmp_trace, iters * sizeof(double), cudaMemcpyDeviceToHost, st));
    int flag = 0;
    KP_TRY_CUDA(cudaMemcpyAsync(&flag, p->d_flag + KP_FLAG_TIMEOUT, sizeof(int), cudaMemcpyDeviceToHost, st));
    KP_TRY_CUDA(cudaStreamSynchronize(st));
    if (flag) return report_timeout(p, st, "a bounded device wait (bulk-copy staging of the interpolation) gave up");
    if (obj_trace)
        for (int k = 0; k < iters; ++k)
            if (!std::isfinite(obj_trace[k])) { set_error("the objective is not finite"); return KP_ENONFINITE; }
    return KP_OK;
}

}  // namespace kp

using namespace kp;

extern "C" {

kp_status kp_make_circulant_preconditioner(kp_plan plan, float* eig_dev, void* stream) {
    KP_RANGE("kp_make_circulant_preconditioner");
    if (!plan) { set_error("null plan"); return KP_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    KP_TRY(circulant_enqueue(plan, st));
    if (eig_dev)
        KP_TRY_CUDA(cudaMemcpyAsync(eig_dev, plan->d_circ_eig, plan->geo.N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    KP_TRY_CUDA(cudaStreamSynchronize(st));
    return KP_OK;
}

kp_status kp_cg_l2_solve(kp_plan plan, const void* y_dev, float lambda, int iters, int circulant, void* x_dev,
                         double* obj_trace, void* stream) {
    KP_RANGE("kp_cg_l2_solve");
    if (!plan || !y_dev || !x_dev) { set_error("null argument"); return KP_EINVAL; }
    if (!plan->traj_set || !plan->maps_set) { set_error("trajectory and maps must be set"); return KP_EINVAL; }
    if (iters < 0) { set_error("iters must be >= 0"); return KP_EINVAL; }
    if (!(lambda >= 0.f) || !std::isfinite(lambda)) { set_error("lambda must be finite and >= 0"); return KP_EINVAL; }
    KP_TRY_CUDA(cudaMemsetAsync(plan->d_flag + KP_FLAG_TIMEOUT, 0, sizeof(int), (cudaStream_t)stream));
    return cg_l2(plan, (const float2*)y_dev, lambda, iters, circulant != 0, (float2*)x_dev, obj_trace, (cudaStream_t)stream);
}

kp_status kp_fista_solve(kp_plan plan, const void* y_dev, kp_reg reg, float lambda, int iters, double lmax, void* x_dev,
                         double* obj_trace, void* stream) {
    KP_RANGE("kp_fista_solve");
    if (!plan || !y_dev || !x_dev) { set_error("null argument"); return KP_EINVAL; }
    if (!plan->traj_set || !plan->maps_set) { set_error("trajectory and maps must be set"); return KP_EINVAL; }
    if (iters < 0) { set_error("iters must be >= 0"); return KP_EINVAL; }
    if (!(lambda >= 0.f) || !std::isfinite(lambda)) { set_error("lambda must be finite and >= 0"); return KP_EINVAL; }
    if (reg != KP_REG_L2 && reg != KP_REG_L1_WAVELET) { set_error("FISTA takes KP_REG_L2 or KP_REG_L1_WAVELET"); return KP_EINVAL; }
    if (reg == KP_REG_L1_WAVELET && plan->P.wavelet_levels < 1) { set_error("l1-wavelet needs wavelet_levels >= 1"); return KP_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    if (!(lmax > 0)) {
        // lambda_max(A^H A) by 30 power iterations from the all-ones image, with a 1 % margin
        KP_TRY(kp_max_eig(plan, nullptr, nullptr, 30, &lmax, stream));
        lmax *= 1.01;
    }
    KP_TRY_CUDA(cudaMemsetAsync(plan->d_flag + KP_FLAG_TIMEOUT, 0, sizeof(int), st));
    return fista(plan, (const float2*)y_dev, (int)reg, lambda, iters, lmax, (float2*)x_dev, obj_trace, st);
}

}  // extern "C"
