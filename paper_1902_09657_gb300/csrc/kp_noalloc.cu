// kp_sense_adjoint_noalloc: the SENSE adjoint x = A^H y without a plan and without any
// device allocation.
//
// Who needs it: callers that reserve all device memory up front and forbid allocation
// afterwards -- for example a scanner-side real-time reconstruction service that sizes its
// memory pool at start-up, or a host application whose device memory is owned by another
// framework's caching allocator.  Such callers cannot let a library call cudaMalloc (or a
// cuFFT planner, which allocates its own work area) in the middle of a reconstruction.
//
// What it computes: the same operator as kp_sense_adjoint (Kaiser-Bessel spreading onto the
// oversampled grid, unnormalised inverse DFT, crop, 1/Phi apodisation, conj(s_c) coil
// combine, N^{-1/2}), with the same float64 grid coordinates and taps.  Because it may not
// create a cuFFT plan, the inverse DFT is evaluated directly, one axis at a time, only at
// the N_d output pixels of each axis; spreading uses global atomics straight into the
// scratch grid.  The results agree with kp_sense_adjoint to float32 rounding (summation
// order differs).
//
// Scratch: one file-scope device array of KP_NOALLOC_SCRATCH_ELEMS complex64 values (4 MiB),
// present on every GPU that loads this library until the process exits.  Its device address
// is looked up (cudaGetSymbolAddress) on every call, with the caller's device current; the
// first call on a device also loads the device code there, so make it before any stream
// capture.  Every call shares the array: the spreading grid is cleared at the start of each
// call, and calls that overlap on the GPU (different streams, or different host threads)
// race on it and must not be issued.
#include "kp_internal.cuh"

#include <cmath>

#define KP_NOALLOC_SCRATCH_ELEMS (1 << 19)

namespace kp {
namespace noalloc {

static __device__ __align__(256) float2 g_scratch[KP_NOALLOC_SCRATCH_ELEMS];

struct Dims {
    int D, C;
    int64_t M;
    int n[MAXD], g[MAXD];
    float beta[MAXD];
    int64_t N, G;
    float rsqrtN;
};

__device__ __forceinline__ int wrapi(int k, int g) { return k < 0 ? k + g : (k >= g ? k - g : k); }

__device__ __forceinline__ float kb4(float u, float beta) {
    float h = 0.5f * u;
    float a = 1.f - h * h;
    return a >= 0.f ? cyl_bessel_i0f(beta * sqrtf(a)) : 0.f;
}

__global__ void k_zero(float2* __restrict__ p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = make_float2(0.f, 0.f);
}

// One thread per sample (caller's order): taps k = ceil(t) - 2 + j, t = f g / n formed in float64.
__global__ void k_spread_atomic(const float* __restrict__ traj, const float2* __restrict__ y, Dims dm,
                                float2* __restrict__ grid) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dm.M) return;
    int idx[MAXD][KW];
    float w[MAXD][KW];
    for (int d = 0; d < dm.D; ++d) {
        const float f = traj[i * dm.D + d];
        const float half = 0.5f * (float)dm.n[d];
        if (!(f >= -half && f <= half)) return;   // out of range or not finite: sample skipped
        float u0;
        const int k0 = grid_tap(f, 1.f, dm.n[d], dm.g[d], &u0);
        for (int j = 0; j < KW; ++j) {
            w[d][j] = kb4(u0 + (float)(KW / 2 - j), dm.beta[d]);
            idx[d][j] = wrapi(k0 + j, dm.g[d]);
        }
    }
    const int taps = dm.D == 2 ? KW * KW : KW * KW * KW;
    for (int c = 0; c < dm.C; ++c) {
        const float2 u = y[(size_t)c * dm.M + i];
        float2* base = grid + (size_t)c * dm.G;
        for (int q = 0; q < taps; ++q) {
            int rem = q;
            float wt = 1.f;
            int64_t off = 0;
            int64_t stride = 1;
            for (int d = dm.D - 1; d >= 0; --d) {
                const int j = rem % KW;
                rem /= KW;
                wt *= w[d][j];
                off += (int64_t)idx[d][j] * stride;
                stride *= dm.g[d];
            }
            atomicAdd(&base[off].x, wt * u.x);
            atomicAdd(&base[off].y, wt * u.y);
        }
    }
}

// Inverse DFT along axis `ax` evaluated at the n_ax centred output positions:
// out[.., j, ..] = sum_k in[.., k, ..] exp(+i 2 pi k (j - n/2) / g).  `shp_in` is the shape
// of the current array per coil (axes after `ax` already reduced to n).
__global__ void k_idft_axis(const float2* __restrict__ in, float2* __restrict__ out, int C, int D, int ax,
                            int s0, int s1, int s2, int g_ax, int n_ax) {
    const int shp[3] = {s0, s1, s2};
    int64_t per_in = 1;
    for (int d = 0; d < D; ++d) per_in *= shp[d];
    const int64_t per_out = per_in / g_ax * n_ax;
    int64_t inner = 1;
    for (int d = ax + 1; d < D; ++d) inner *= shp[d];
    const int64_t total = (int64_t)C * per_out;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = o / per_out;
        const int64_t r = o % per_out;
        const int64_t lo = r % inner;
        const int64_t rest = r / inner;
        const int j = (int)(rest % n_ax);
        const int64_t hi = rest / n_ax;
        const int nc = j - n_ax / 2;
        const float2* src = in + c * per_in + hi * (int64_t)g_ax * inner + lo;
        float2 acc = make_float2(0.f, 0.f);
        for (int k = 0; k < g_ax; ++k) {
            int m = (int)(((int64_t)k * nc) % g_ax);
            if (m < 0) m += g_ax;
            float s, cs;
            sincospif(2.0f * (float)m / (float)g_ax, &s, &cs);
            const float2 v = src[(int64_t)k * inner];
            acc.x += v.x * cs - v.y * s;
            acc.y += v.x * s + v.y * cs;
        }
        out[o] = acc;
    }
}

// x[j] = N^{-1/2} prod_d 1/Phi_d(n_d) sum_c conj(s_c[j]) img_c[j]
__global__ void k_combine(const float2* __restrict__ img, const float2* __restrict__ maps, Dims dm,
                          float2* __restrict__ x) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= dm.N) return;
    int64_t r = j;
    double a = 1.0;
    const double pi = 3.14159265358979323846;
    for (int d = dm.D - 1; d >= 0; --d) {
        const int jd = (int)(r % dm.n[d]);
        r /= dm.n[d];
        const double nn = (double)(jd - dm.n[d] / 2);
        const double beta = (double)dm.beta[d];
        const double z2 = beta * beta - (pi * KW * nn / dm.g[d]) * (pi * KW * nn / dm.g[d]);
        double phi;
        if (z2 > 0) { const double z = sqrt(z2); phi = KW * sinh(z) / z; }
        else if (z2 < 0) { const double z = sqrt(-z2); phi = KW * sin(z) / z; }
        else phi = KW;
        a *= (double)(float)(1.0 / phi);
    }
    float2 acc = make_float2(0.f, 0.f);
    for (int c = 0; c < dm.C; ++c) {
        const float2 v = img[(size_t)c * dm.N + j];
        const float2 s = maps[(size_t)c * dm.N + j];
        acc.x += s.x * v.x + s.y * v.y;
        acc.y += s.x * v.y - s.y * v.x;
    }
    const float sc = (float)a * dm.rsqrtN;
    x[j] = make_float2(acc.x * sc, acc.y * sc);
}

// Device address of the scratch array on the current device, looked up on every call: the
// lookup allocates nothing, and a cached address would go stale after cudaDeviceReset or a
// re-created primary context.  The first lookup on a device also loads this library's device
// code there, which is why the first call should not be made during a stream capture.
static kp_status scratch_address(float2** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
        set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        return KP_ECUDA;
    }
    *out = (float2*)p;
    return KP_OK;
}

}  // namespace noalloc
}  // namespace kp

using namespace kp;

extern "C" kp_status kp_sense_adjoint_noalloc(const kp_params* params, const float* traj_dev, const void* maps_dev,
                                              const void* y_dev, void* x_dev, void* stream) {
    KP_RANGE("kp_sense_adjoint_noalloc");
    using namespace kp::noalloc;
    if (!params || !traj_dev || !maps_dev || !y_dev || !x_dev) { set_error("null argument"); return KP_EINVAL; }
    const int D = params->ndim;
    if (D != 2 && D != 3) { set_error("ndim must be 2 or 3"); return KP_EINVAL; }
    if (params->kernel_width != KW) { set_error("kernel_width must be 4"); return KP_EINVAL; }
    if (params->ncoils < 1 || params->nsamples < 1) { set_error("ncoils and nsamples must be >= 1"); return KP_EINVAL; }
    if (!(params->oversamp >= 1.0f && params->oversamp <= 4.0f)) { set_error("oversamp must be in [1, 4]"); return KP_EINVAL; }
    Dims dm{};
    dm.D = D;
    dm.C = params->ncoils;
    dm.M = params->nsamples;
    dm.N = 1;
    dm.G = 1;
    for (int d = 0; d < MAXD; ++d) { dm.n[d] = 1; dm.g[d] = 1; dm.beta[d] = 0.f; }
    for (int d = 0; d < D; ++d) {
        if (params->img[d] < 8 || params->img[d] > 4096) { set_error("image sizes must be in [8, 4096]"); return KP_EINVAL; }
        const int n = (int)params->img[d];
        int g = (int)std::ceil((double)params->oversamp * n - 1e-9);
        g += g & 1;
        const double a = (double)g / n;
        const double b2 = (KW / a) * (KW / a) * (a - 0.5) * (a - 0.5) - 0.8;
        if (b2 <= 0) { set_error("oversampling too small for a Kaiser-Bessel width of 4"); return KP_EINVAL; }
        dm.n[d] = n;
        dm.g[d] = g;
        dm.beta[d] = (float)(3.14159265358979323846 * std::sqrt(b2));
        dm.N *= n;
        dm.G *= g;
    }
    dm.rsqrtN = (float)(1.0 / std::sqrt((double)dm.N));
    // scratch: the C x G spreading grid, then a ping-pong pair for the per-axis inverse DFTs
    int64_t stage = dm.G, peak = 0;
    for (int ax = D - 1; ax >= 0; --ax) {
        const int64_t next = stage / dm.g[ax] * dm.n[ax];
        peak = std::max<int64_t>(peak, stage + next);
        stage = next;
    }
    const int64_t need = (int64_t)dm.C * peak;
    if (need > KP_NOALLOC_SCRATCH_ELEMS) {
        set_error("problem too large for the allocation-free path: needs " + std::to_string(need) +
                  " complex scratch values, the fixed array holds " + std::to_string(KP_NOALLOC_SCRATCH_ELEMS) +
                  " (C x (G + G n_last / g_last) must fit)");
        return KP_EINVAL;
    }
    float2* scratch = nullptr;
    KP_TRY(scratch_address(&scratch));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t CG = (int64_t)dm.C * dm.G;
    k_zero<<<(unsigned)std::min<int64_t>((CG + 255) / 256, 4096), 256, 0, st>>>(scratch, CG);
    KP_LAUNCH_CHECK();
    k_spread_atomic<<<(unsigned)((dm.M + 127) / 128), 128, 0, st>>>(traj_dev, (const float2*)y_dev, dm, scratch);
    KP_LAUNCH_CHECK();
    // inverse DFT axis by axis (last axis first).  Region A = [0, C G) holds the grid; pass
    // outputs alternate between region B = [C G, C (G + G_1)) and A, and each fits its region.
    int shp[3] = {dm.g[0], dm.g[1], dm.g[2]};
    float2* const bufA = scratch;
    float2* const bufB = scratch + CG;
    float2* cur = bufA;
    for (int ax = D - 1; ax >= 0; --ax) {
        int64_t per_out = 1;
        for (int d = 0; d < D; ++d) per_out *= (d == ax ? dm.n[d] : shp[d]);
        const int64_t tot = (int64_t)dm.C * per_out;
        float2* dst = cur == bufA ? bufB : bufA;
        k_idft_axis<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 8192), 256, 0, st>>>(
            cur, dst, dm.C, D, ax, shp[0], shp[1], shp[2], dm.g[ax], dm.n[ax]);
        KP_LAUNCH_CHECK();
        shp[ax] = dm.n[ax];
        cur = dst;
    }
    k_combine<<<(unsigned)((dm.N + 255) / 256), 256, 0, st>>>(cur, (const float2*)maps_dev, dm, (float2*)x_dev);
    KP_LAUNCH_CHECK();
    return KP_OK;
}
