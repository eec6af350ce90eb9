// Periodised multilevel Daubechies-4 transform W (Sec. 2: W unitary; Sec. 6: Daubechies-4)
// and the l1-wavelet prox W^H S_t(W z) of the PDHG primal step (Sec. 4.1).
//
// One kernel per level and direction.  A CTA owns a tile of T^D output positions, stages the
// periodic input footprint in shared memory and filters it axis by axis there, so one launch
// does every axis of a level.  Forward level l reads the level-(l-1) approximation and writes
// its 2^D - 1 detail subbands to the coefficient image at their Mallat positions (the last
// level also writes its approximation there); the other approximations go to two small
// ping-pong buffers.  Inverse level l reads the level-l approximation and the details and
// writes the level-(l-1) approximation (or the image at l = 0).  The soft threshold S_t is
// applied as the forward kernels write the coefficients, and PDHG's extrapolation
// xbar = x + theta (x - x_old) is fused into the last inverse level, so the whole prox is
// 2 L launches.
//
// Filters: analysis a[k] = sum_n h[n] x[2k+n], d[k] = sum_n g[n] x[2k+n] (indices mod the
// block length), g[n] = (-1)^n h[7-n]; synthesis is the transpose.
#include "kp_internal.cuh"

namespace kp {

__constant__ float c_wh[8];
__constant__ float c_wg[8];

kp_status upload_wavelet_filter(const float h[8]) {
    float g[8];
    for (int n = 0; n < 8; ++n) g[n] = (n & 1 ? -1.f : 1.f) * h[7 - n];
    KP_TRY_CUDA(cudaMemcpyToSymbol(c_wh, h, 8 * sizeof(float)));
    KP_TRY_CUDA(cudaMemcpyToSymbol(c_wg, g, 8 * sizeof(float)));
    return KP_OK;
}

struct View {            // strided complex image view: element i at p[sum_d i_d * s_d]
    float2* p;
    int64_t s[MAXD];
};

struct LevelArgs {
    View src, dst;       // src: approximation in; dst: approximation out (when not coef)
    View coef;           // coefficient image (Mallat layout, full size)
    int b[MAXD];         // block (input) size per axis for forward, output size for inverse
    int tiles[MAXD];     // tiles per axis
    int lev_last;        // forward: write LL to coef; inverse: read LL from coef
    int lev_first;       // inverse: output is the image (extrapolation / plain store)
    const float* sched;  // soft threshold tau_k * lambda and theta_k (null: none)
    const int* iter;
    float lambda;
    float2* x;           // extrapolation targets (inverse, first level, prox mode)
    float2* xbar;
};

template <int D>
__device__ __forceinline__ int64_t voff(const View& v, const int* i) {
    int64_t o = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) o += (int64_t)i[d] * v.s[d];
    return o;
}

// Filter one axis of a shared-memory block: in has extents ein[], out has extents eout[]
// (equal except along `ax`).  Forward: out[.., q, ..] for q < K is a[k0 + q], for q >= K is
// d[k0 + q - K], from in[.., 2q' + n, ..].
template <int D, int K>
__device__ __forceinline__ void fwd_axis(const float2* __restrict__ in, const int* ein, float2* __restrict__ out,
                                         const int* eout, int ax) {
    int tot = 1;
#pragma unroll
    for (int d = 0; d < D; ++d) tot *= eout[d];
    for (int o = threadIdx.x; o < tot; o += blockDim.x) {
        int idx[D];
        int r = o;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { idx[d] = r % eout[d]; r /= eout[d]; }
        const int q = idx[ax];
        const bool det = q >= K;
        const int k = det ? q - K : q;
        int base = 0, stride = 1, sax = 1;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            if (d == ax) sax = stride;
            base += (d == ax ? 2 * k : idx[d]) * stride;
            stride *= ein[d];
        }
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const float c = det ? c_wg[n] : c_wh[n];
            const float2 v = in[base + n * sax];
            acc.x = fmaf(c, v.x, acc.x);
            acc.y = fmaf(c, v.y, acc.y);
        }
        out[o] = acc;
    }
}

// Inverse along one axis: in holds [a (K+4) | d (K+4)] coefficients for k = kb .. kb+K+3,
// out holds 2K outputs for j = 2 kb + 8 .. (so that j - n for n < 8 stays >= 2 kb).
template <int D, int K>
__device__ __forceinline__ void inv_axis(const float2* __restrict__ in, const int* ein, float2* __restrict__ out,
                                         const int* eout, int ax) {
    int tot = 1;
#pragma unroll
    for (int d = 0; d < D; ++d) tot *= eout[d];
    constexpr int E = K + 4;
    for (int o = threadIdx.x; o < tot; o += blockDim.x) {
        int idx[D];
        int r = o;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { idx[d] = r % eout[d]; r /= eout[d]; }
        const int jl = idx[ax];            // output j = j0 + jl, j0 = 2 kb + 8
        int base = 0, stride = 1, sax = 1;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            if (d == ax) sax = stride;
            base += (d == ax ? 0 : idx[d]) * stride;
            stride *= ein[d];
        }
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int n = (jl & 1) + 2 * m;
            const int kl = (jl + 8 - n) >> 1;    // (j - n)/2 - kb, in [0, K+4)
            const float2 av = in[base + kl * sax];
            const float2 dv = in[base + (E + kl) * sax];
            acc.x = fmaf(c_wh[n], av.x, fmaf(c_wg[n], dv.x, acc.x));
            acc.y = fmaf(c_wh[n], av.y, fmaf(c_wg[n], dv.y, acc.y));
        }
        out[o] = acc;
    }
}

__device__ __forceinline__ float2 soft(float2 c, float t) {
    const float m = sqrtf(c.x * c.x + c.y * c.y);
    const float s = m > t ? 1.f - t / m : 0.f;
    return make_float2(c.x * s, c.y * s);
}

template <int D, int T>
__global__ void __launch_bounds__(256) k_dwt_fwd_level(LevelArgs a) {
    extern __shared__ float2 sm[];
    constexpr int EI = 2 * T + 6;
    int tc[D];
    {
        int r = blockIdx.x;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { tc[d] = r % a.tiles[d]; r /= a.tiles[d]; }
    }
    int k0[D], h[D];
#pragma unroll
    for (int d = 0; d < D; ++d) { k0[d] = tc[d] * T; h[d] = a.b[d] / 2; }
    // stage the periodic input footprint [2 k0, 2 k0 + 2T + 6) per axis
    int ein[D];
    int tot = 1;
#pragma unroll
    for (int d = 0; d < D; ++d) { ein[d] = EI; tot *= EI; }
    float2* buf0 = sm;
    float2* buf1 = sm + tot;
    for (int o = threadIdx.x; o < tot; o += blockDim.x) {
        int i[D];
        int r = o;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            int l = r % EI;
            r /= EI;
            i[d] = (2 * k0[d] + l) % a.b[d];
        }
        buf0[o] = a.src.p[voff<D>(a.src, i)];
    }
    __syncthreads();
    // filter axis by axis, last axis first
    int ecur[D];
#pragma unroll
    for (int d = 0; d < D; ++d) ecur[d] = EI;
    float2* in = buf0;
    float2* out = buf1;
#pragma unroll
    for (int ax = D - 1; ax >= 0; --ax) {
        int eout[D];
#pragma unroll
        for (int d = 0; d < D; ++d) eout[d] = d == ax ? 2 * T : ecur[d];
        fwd_axis<D, T>(in, ecur, out, eout, ax);
        __syncthreads();
#pragma unroll
        for (int d = 0; d < D; ++d) ecur[d] = eout[d];
        float2* t = in;
        in = out;
        out = t;
    }
    // in now holds (2T)^D values: per axis q < T -> a[k0+q], q >= T -> d[k0+q-T]
    const float thr = a.sched ? a.sched[3 * (*a.iter) + 1] * a.lambda : 0.f;
    int tot2 = 1;
#pragma unroll
    for (int d = 0; d < D; ++d) tot2 *= 2 * T;
    for (int o = threadIdx.x; o < tot2; o += blockDim.x) {
        int q[D];
        int r = o;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { q[d] = r % (2 * T); r /= 2 * T; }
        bool ok = true, all_a = true;
        int pos[D], posll[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const bool det = q[d] >= T;
            const int k = k0[d] + (det ? q[d] - T : q[d]);
            if (k >= h[d]) ok = false;
            if (det) all_a = false;
            pos[d] = det ? h[d] + k : k;
            posll[d] = k;
        }
        if (!ok) continue;
        float2 v = in[o];
        if (all_a && !a.lev_last) {
            a.dst.p[voff<D>(a.dst, posll)] = v;
        } else {
            if (a.sched) v = soft(v, thr);
            a.coef.p[voff<D>(a.coef, pos)] = v;
        }
    }
}

template <int D, int T>
__global__ void __launch_bounds__(256) k_dwt_inv_level(LevelArgs a) {
    extern __shared__ float2 sm[];
    constexpr int E = T + 4;      // coefficients per subband per axis
    int tc[D];
    {
        int r = blockIdx.x;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { tc[d] = r % a.tiles[d]; r /= a.tiles[d]; }
    }
    // output j in [2 T tc, 2 T tc + 2T); coefficients k in [kb, kb + T + 4), kb = T tc - 4
    int kb[D], hh[D];
#pragma unroll
    for (int d = 0; d < D; ++d) { kb[d] = T * tc[d] - 4; hh[d] = a.b[d] / 2; }
    int tot = 1;
#pragma unroll
    for (int d = 0; d < D; ++d) tot *= 2 * E;
    float2* buf0 = sm;
    float2* buf1 = sm + tot;
    for (int o = threadIdx.x; o < tot; o += blockDim.x) {
        int r = o;
        bool all_a = true;
        int pos[D], posll[D];
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            const int l = r % (2 * E);
            r /= 2 * E;
            const bool det = l >= E;
            int k = kb[d] + (det ? l - E : l);
            k = ((k % hh[d]) + hh[d]) % hh[d];
            if (det) all_a = false;
            pos[d] = det ? hh[d] + k : k;
            posll[d] = k;
        }
        float2 v;
        if (all_a && !a.lev_last) v = a.src.p[voff<D>(a.src, posll)];
        else v = a.coef.p[voff<D>(a.coef, pos)];
        buf0[o] = v;
    }
    __syncthreads();
    int ecur[D];
#pragma unroll
    for (int d = 0; d < D; ++d) ecur[d] = 2 * E;
    float2* in = buf0;
    float2* out = buf1;
#pragma unroll
    for (int ax = D - 1; ax >= 0; --ax) {
        int eout[D];
#pragma unroll
        for (int d = 0; d < D; ++d) eout[d] = d == ax ? 2 * T : ecur[d];
        inv_axis<D, T>(in, ecur, out, eout, ax);
        __syncthreads();
#pragma unroll
        for (int d = 0; d < D; ++d) ecur[d] = eout[d];
        float2* t = in;
        in = out;
        out = t;
    }
    // inv_axis produced outputs for j = 2 kb + 8 + jl = 2 T tc + jl
    const float th = (a.lev_first && a.x) ? a.sched[3 * (*a.iter) + 2] : 0.f;
    int tot2 = 1;
#pragma unroll
    for (int d = 0; d < D; ++d) tot2 *= 2 * T;
    for (int o = threadIdx.x; o < tot2; o += blockDim.x) {
        int jl[D], j[D];
        int r = o;
        bool ok = true;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { jl[d] = r % (2 * T); r /= 2 * T; }
#pragma unroll
        for (int d = 0; d < D; ++d) {
            j[d] = 2 * T * tc[d] + jl[d];
            if (j[d] >= a.b[d]) ok = false;
        }
        if (!ok) continue;
        const float2 v = in[o];
        const int64_t off = voff<D>(a.dst, j);
        if (a.lev_first && a.x) {
            const float2 xo = a.x[off];
            a.xbar[off] = make_float2(v.x + th * (v.x - xo.x), v.y + th * (v.y - xo.y));
            a.x[off] = v;
        } else {
            a.dst.p[off] = v;
        }
    }
}

static inline int wt_tile(int D) { return D == 2 ? 16 : 8; }

static View full_view(float2* p, const Geom& g) {
    View v{};
    v.p = p;
    int64_t s = 1;
    for (int d = g.D - 1; d >= 0; --d) { v.s[d] = s; s *= g.n[d]; }
    return v;
}

static View dense_view(float2* p, const int* dims, int D) {
    View v{};
    v.p = p;
    int64_t s = 1;
    for (int d = D - 1; d >= 0; --d) { v.s[d] = s; s *= dims[d]; }
    return v;
}

template <int D, int T>
static kp_status launch_fwd(const LevelArgs& a, int nblocks, cudaStream_t st) {
    constexpr int EI = 2 * T + 6;
    size_t tot = 1, tot1 = 1;
    for (int d = 0; d < D; ++d) { tot *= EI; tot1 *= (d == D - 1 ? 2 * T : EI); }
    const size_t smem = (tot + tot1) * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        KP_TRY_CUDA(cudaFuncSetAttribute(k_dwt_fwd_level<D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr = true;
    }
    k_dwt_fwd_level<D, T><<<nblocks, 256, smem, st>>>(a);
    KP_LAUNCH_CHECK();
    return KP_OK;
}

template <int D, int T>
static kp_status launch_inv(const LevelArgs& a, int nblocks, cudaStream_t st) {
    constexpr int E = T + 4;
    size_t tot = 1, tot1 = 1;
    for (int d = 0; d < D; ++d) { tot *= 2 * E; tot1 *= (d == D - 1 ? 2 * T : 2 * E); }
    const size_t smem = (tot + tot1) * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        KP_TRY_CUDA(cudaFuncSetAttribute(k_dwt_inv_level<D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr = true;
    }
    k_dwt_inv_level<D, T><<<nblocks, 256, smem, st>>>(a);
    KP_LAUNCH_CHECK();
    return KP_OK;
}

// Forward W (coefficients in Mallat layout into `coef`), optionally soft-thresholded at
// tau_k lambda (prox mode, sched != null).
static kp_status wavelet_forward(kp_plan p, const float2* in, float2* coef, const float* sched, float lambda,
                                 cudaStream_t st) {
    const Geom& g = p->geo;
    const int L = p->P.wavelet_levels;
    const int T = wt_tile(g.D);
    float2* ll[2] = {p->d_wl0, p->d_wl1};
    mark(p, PH_DWT_FWD, st);
    for (int lev = 0; lev < L; ++lev) {
        LevelArgs a{};
        int bdim[MAXD], hdim[MAXD];
        int nb = 1;
        for (int d = 0; d < g.D; ++d) {
            bdim[d] = g.n[d] >> lev;
            hdim[d] = bdim[d] / 2;
            a.b[d] = bdim[d];
            a.tiles[d] = (hdim[d] + T - 1) / T;
            nb *= a.tiles[d];
        }
        a.src = lev == 0 ? full_view(const_cast<float2*>(in), g) : dense_view(ll[(lev - 1) & 1], bdim, g.D);
        a.dst = dense_view(ll[lev & 1], hdim, g.D);
        a.coef = full_view(coef, g);
        a.lev_last = lev == L - 1;
        a.sched = sched;
        a.iter = p->d_iter;
        a.lambda = lambda;
        if (g.D == 2) KP_TRY((launch_fwd<2, 16>(a, nb, st)));
        else KP_TRY((launch_fwd<3, 8>(a, nb, st)));
        p->launches += 1;
    }
    return KP_OK;
}

// Inverse W from Mallat-layout coefficients; in prox mode (x != null) the last level writes
// x_new and the extrapolation xbar = x_new + theta_k (x_new - x).
static kp_status wavelet_inverse(kp_plan p, const float2* coef, float2* out, float2* x, float2* xbar,
                                 const float* sched, cudaStream_t st) {
    const Geom& g = p->geo;
    const int L = p->P.wavelet_levels;
    const int T = wt_tile(g.D);
    float2* ll[2] = {p->d_wl0, p->d_wl1};
    mark(p, PH_DWT_INV, st);
    for (int lev = L - 1; lev >= 0; --lev) {
        LevelArgs a{};
        int bdim[MAXD], hdim[MAXD];
        int nb = 1;
        for (int d = 0; d < g.D; ++d) {
            bdim[d] = g.n[d] >> lev;
            hdim[d] = bdim[d] / 2;
            a.b[d] = bdim[d];
            a.tiles[d] = (bdim[d] + 2 * T - 1) / (2 * T);
            nb *= a.tiles[d];
        }
        a.src = dense_view(ll[lev & 1], hdim, g.D);
        a.coef = full_view(const_cast<float2*>(coef), g);
        a.dst = lev == 0 ? full_view(x ? x : out, g) : dense_view(ll[(lev - 1) & 1], bdim, g.D);
        a.lev_last = lev == L - 1;
        a.lev_first = lev == 0;
        a.sched = sched;
        a.iter = p->d_iter;
        a.x = (lev == 0) ? x : nullptr;
        a.xbar = (lev == 0) ? xbar : nullptr;
        if (g.D == 2) KP_TRY((launch_inv<2, 16>(a, nb, st)));
        else KP_TRY((launch_inv<3, 8>(a, nb, st)));
        p->launches += 1;
    }
    return KP_OK;
}

kp_status wavelet_apply(kp_plan p, const float2* in, float2* out, bool forward, cudaStream_t st) {
    if (forward) {
        if (in == out) {
            // the level kernels read the image while writing coefficients: stage a copy
            KP_TRY_CUDA(cudaMemcpyAsync(p->d_w, in, p->geo.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
            in = p->d_w;
        }
        return wavelet_forward(p, in, out, nullptr, 0.f, st);
    }
    if (in == out) {
        KP_TRY_CUDA(cudaMemcpyAsync(p->d_w, in, p->geo.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        in = p->d_w;
    }
    return wavelet_inverse(p, in, out, nullptr, nullptr, nullptr, st);
}

// PDHG l1-wavelet prox with extrapolation: z -> coefficients (thresholded) -> x_new, xbar.
kp_status wavelet_prox_extrap(kp_plan p, float lambda, cudaStream_t st) {
    KP_TRY(wavelet_forward(p, p->d_z, p->d_w, p->d_sched, lambda, st));
    KP_TRY(wavelet_inverse(p, p->d_w, nullptr, p->d_x, p->d_xbar, p->d_sched, st));
    return KP_OK;
}

}  // namespace kp
