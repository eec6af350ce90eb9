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
// xbar = x + theta (x - x_old) is fused into the last inverse level.  Inside a PDHG iteration
// the level passes run in one persistent cooperative kernel (k_primal_fused, end of file),
// separated by grid barriers; the standalone level kernels serve kp_wavelet and the batched
// iteration (several cases at once, where one cooperative grid per case cannot co-reside).
//
// Filters: analysis a[k] = sum_n h[n] x[2k+n], d[k] = sum_n g[n] x[2k+n] (indices mod the
// block length), g[n] = (-1)^n h[7-n]; synthesis is the transpose.
#include "kp_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>

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
    float2* fgrid;       // when set (inverse, first level): write s_c xbar / Phi into the forward grid
    const void* maps;
    const float* apod;
    Geom geo;
    int tiles_total;     // number of tiles of the level
};

template <int D>
__device__ __forceinline__ int64_t voff(const View& v, const int* i) {
    int64_t o = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) o += (int64_t)i[d] * v.s[d];
    return o;
}

// Filter one axis of a shared-memory block with compile-time extents: the input block has
// extents (I0, I1, I2) (the last D used); the output equals it except along AX, which becomes
// 2K.  Forward: out q < K is a[k0 + q], q >= K is d[k0 + q - K], from in[2 (q mod K) + n].
template <int D, int K, int AX, int I0, int I1, int I2>
__device__ __forceinline__ void fwd_axis_c(const float2* __restrict__ in, float2* __restrict__ out) {
    constexpr int EI[3] = {I0, I1, I2};
    constexpr int O0 = AX == 0 ? 2 * K : I0, O1 = AX == 1 ? 2 * K : I1, O2 = AX == 2 ? 2 * K : I2;
    constexpr int EO[3] = {O0, O1, O2};
    constexpr int TOT = D == 2 ? O0 * O1 : O0 * O1 * O2;
    constexpr int SAX = AX == D - 1 ? 1 : (AX == D - 2 ? EI[D - 1] : EI[1] * EI[2]);
    for (int o = threadIdx.x; o < TOT; o += blockDim.x) {
        int idx[3];
        int r = o;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { idx[d] = r % EO[d]; r /= EO[d]; }
        const int q = idx[AX];
        const bool det = q >= K;
        const int k = det ? q - K : q;
        int base = 0, stride = 1;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            base += (d == AX ? 2 * k : idx[d]) * stride;
            stride *= EI[d];
        }
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const float c = det ? c_wg[n] : c_wh[n];
            const float2 v = in[base + n * SAX];
            acc.x = fmaf(c, v.x, acc.x);
            acc.y = fmaf(c, v.y, acc.y);
        }
        out[o] = acc;
    }
}

// Inverse along AX: the input holds [a (K+4) | d (K+4)] coefficients per axis position for
// k = kb .. kb+K+3; the output holds 2K values for j = 2 kb + 8 ...
template <int D, int K, int AX, int I0, int I1, int I2>
__device__ __forceinline__ void inv_axis_c(const float2* __restrict__ in, float2* __restrict__ out) {
    constexpr int EI[3] = {I0, I1, I2};
    constexpr int O0 = AX == 0 ? 2 * K : I0, O1 = AX == 1 ? 2 * K : I1, O2 = AX == 2 ? 2 * K : I2;
    constexpr int EO[3] = {O0, O1, O2};
    constexpr int TOT = D == 2 ? O0 * O1 : O0 * O1 * O2;
    constexpr int SAX = AX == D - 1 ? 1 : (AX == D - 2 ? EI[D - 1] : EI[1] * EI[2]);
    constexpr int E = K + 4;
    for (int o = threadIdx.x; o < TOT; o += blockDim.x) {
        int idx[3];
        int r = o;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { idx[d] = r % EO[d]; r /= EO[d]; }
        const int jl = idx[AX];
        int base = 0, stride = 1;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            base += (d == AX ? 0 : idx[d]) * stride;
            stride *= EI[d];
        }
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int n = (jl & 1) + 2 * m;
            const int kl = (jl + 8 - n) >> 1;
            const float2 av = in[base + kl * SAX];
            const float2 dv = in[base + (E + kl) * SAX];
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
__device__ __forceinline__ void fwd_level_tile(const LevelArgs& a, int tile, float2* sm) {
    constexpr int EI = 2 * T + 6;
    int tc[D];
    {
        int r = tile;
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
    // filter axis by axis, last axis first (buf0 -> buf1 -> buf0 [-> buf1 in 3D])
    constexpr int T2 = 2 * T;
    float2* in;
    if (D == 2) {
        fwd_axis_c<D, T, 1, EI, EI, 1>(buf0, buf1);
        __syncthreads();
        fwd_axis_c<D, T, 0, EI, T2, 1>(buf1, buf0);
        __syncthreads();
        in = buf0;
    } else {
        fwd_axis_c<D, T, 2, EI, EI, EI>(buf0, buf1);
        __syncthreads();
        fwd_axis_c<D, T, 1, EI, EI, T2>(buf1, buf0);
        __syncthreads();
        fwd_axis_c<D, T, 0, EI, T2, T2>(buf0, buf1);
        __syncthreads();
        in = buf1;
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
    __syncthreads();   // shared memory is reused by the next tile
}

template <int D, int T, typename MT>
__device__ __forceinline__ void inv_level_tile(const LevelArgs& a, int tile, float2* sm) {
    constexpr int E = T + 4;      // coefficients per subband per axis
    int tc[D];
    {
        int r = tile;
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
    constexpr int T2 = 2 * T, E2 = 2 * E;
    float2* in;
    if (D == 2) {
        inv_axis_c<D, T, 1, E2, E2, 1>(buf0, buf1);
        __syncthreads();
        inv_axis_c<D, T, 0, E2, T2, 1>(buf1, buf0);
        __syncthreads();
        in = buf0;
    } else {
        inv_axis_c<D, T, 2, E2, E2, E2>(buf0, buf1);
        __syncthreads();
        inv_axis_c<D, T, 1, E2, E2, T2>(buf1, buf0);
        __syncthreads();
        inv_axis_c<D, T, 0, E2, T2, T2>(buf0, buf1);
        __syncthreads();
        in = buf1;
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
        if (a.lev_first && a.x && !KP_INB(13, off, a.geo.N)) continue;
        if (a.lev_first && a.x) {
            const float2 xo = a.x[off];
            const float2 xb = make_float2(v.x + th * (v.x - xo.x), v.y + th * (v.y - xo.y));
            a.xbar[off] = xb;
            a.x[off] = v;
            if (a.fgrid) pre_pixel<D, MT>(a.fgrid, (const MT*)a.maps, a.apod, a.geo, off, xb);
        } else {
            a.dst.p[off] = v;
        }
    }
    __syncthreads();   // shared memory is reused by the next tile
}

template <int D, int T>
__global__ void __launch_bounds__(256) k_dwt_fwd_level(LevelArgs a) {
    extern __shared__ float2 sm[];
    fwd_level_tile<D, T>(a, blockIdx.x, sm);
}

template <int D, int T>
__global__ void __launch_bounds__(256) k_dwt_inv_level(LevelArgs a) {
    extern __shared__ float2 sm[];
    inv_level_tile<D, T, float2>(a, blockIdx.x, sm);
}

template <int D, int T, typename MT>
__global__ void __launch_bounds__(256) k_dwt_inv_level_t(LevelArgs a) {
    extern __shared__ float2 sm[];
    inv_level_tile<D, T, MT>(a, blockIdx.x, sm);
}

// The level kernels over the cases of a batch (block -> case as in the other batched launches).
template <int D, int T>
__global__ void __launch_bounds__(256) k_dwt_fwd_level_b(const LevelArgs* __restrict__ cs, const int* __restrict__ boff,
                                                         int ncase) {
    extern __shared__ float2 sm[];
    const int c = batch_case(boff, ncase, (int)blockIdx.x);
    fwd_level_tile<D, T>(cs[c], (int)blockIdx.x - boff[c], sm);
}

template <int D, int T, typename MT>
__global__ void __launch_bounds__(256) k_dwt_inv_level_b(const LevelArgs* __restrict__ cs, const int* __restrict__ boff,
                                                         int ncase) {
    extern __shared__ float2 sm[];
    const int c = batch_case(boff, ncase, (int)blockIdx.x);
    inv_level_tile<D, T, MT>(cs[c], (int)blockIdx.x - boff[c], sm);
}

static inline int wt_tile(int D) { return D == 2 ? 16 : 8; }

template <int D, int T, typename MT>
static kp_status launch_inv_t(const LevelArgs& a, int nblocks, cudaStream_t st) {
    constexpr int E = T + 4;
    size_t tot = 1, tot1 = 1;
    for (int d = 0; d < D; ++d) { tot *= 2 * E; tot1 *= (d == D - 1 ? 2 * T : 2 * E); }
    const size_t smem = (tot + tot1) * sizeof(float2);
    static PerDeviceOnce attr;
    if (attr.first()) KP_TRY_CUDA(cudaFuncSetAttribute(k_dwt_inv_level_t<D, T, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    k_dwt_inv_level_t<D, T, MT><<<nblocks, 256, smem, st>>>(a);
    KP_LAUNCH_CHECK();
    return KP_OK;
}

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
    static PerDeviceOnce attr;
    if (attr.first()) KP_TRY_CUDA(cudaFuncSetAttribute(k_dwt_fwd_level<D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
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
    static PerDeviceOnce attr;
    if (attr.first()) KP_TRY_CUDA(cudaFuncSetAttribute(k_dwt_inv_level<D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    k_dwt_inv_level<D, T><<<nblocks, 256, smem, st>>>(a);
    KP_LAUNCH_CHECK();
    return KP_OK;
}

// Forward W (coefficients in Mallat layout into `coef`), optionally soft-thresholded at
// tau_k lambda (prox mode, sched != null).
// Forward W (coefficients in Mallat layout into `coef`), no threshold.
static kp_status wavelet_forward(kp_plan p, const float2* in, float2* coef, cudaStream_t st) {
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
        a.iter = p->d_iter;
        if (g.D == 2) KP_TRY((launch_fwd<2, 16>(a, nb, st)));
        else KP_TRY((launch_fwd<3, 8>(a, nb, st)));
        p->launches += 1;
    }
    return KP_OK;
}

// Inverse W from Mallat-layout coefficients.
static kp_status wavelet_inverse(kp_plan p, const float2* coef, float2* out, cudaStream_t st) {
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
        a.dst = lev == 0 ? full_view(out, g) : dense_view(ll[(lev - 1) & 1], bdim, g.D);
        a.lev_last = lev == L - 1;
        a.lev_first = lev == 0;
        a.iter = p->d_iter;
        if (g.D == 2) KP_TRY((launch_inv<2, 16>(a, nb, st)));
        else KP_TRY((launch_inv<3, 8>(a, nb, st)));
        p->launches += 1;
    }
    return KP_OK;
}

// l1-wavelet prox of the PDHG primal step with the standalone level kernels (for runs in
// which several plans share the GPU concurrently, where a cooperative grid-wide kernel per
// plan is not used): z -> thresholded coefficients -> x_new, xbar and the forward grid.
kp_status wavelet_prox_levels(kp_plan p, float lambda, cudaStream_t st) {
    const Geom& g = p->geo;
    const int L = p->P.wavelet_levels;
    const int T = wt_tile(g.D);
    float2* ll[2] = {p->d_wl0, p->d_wl1};
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
        a.src = lev == 0 ? full_view(p->d_z, g) : dense_view(ll[(lev - 1) & 1], bdim, g.D);
        a.dst = dense_view(ll[lev & 1], hdim, g.D);
        a.coef = full_view(p->d_w, g);
        a.lev_last = lev == L - 1;
        a.sched = p->d_sched;
        a.iter = p->d_iter;
        a.lambda = lambda;
        if (g.D == 2) KP_TRY((launch_fwd<2, 16>(a, nb, st)));
        else KP_TRY((launch_fwd<3, 8>(a, nb, st)));
        p->launches += 1;
    }
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
        a.coef = full_view(p->d_w, g);
        a.dst = lev == 0 ? full_view(p->d_x, g) : dense_view(ll[(lev - 1) & 1], bdim, g.D);
        a.lev_last = lev == L - 1;
        a.lev_first = lev == 0;
        a.sched = p->d_sched;
        a.iter = p->d_iter;
        if (lev == 0) {
            a.x = p->d_x;
            a.xbar = p->d_xbar;
            a.fgrid = p->fft3 ? nullptr : p->d_grid;      // the own FFT forms the pre-step itself
            a.maps = p->d_maps;
            a.apod = p->d_apod;
            a.geo = g;
        }
        const kp_cdtype mt = p->maps_t;
        if (g.D == 2) {
            if (mt == KP_C64) KP_TRY((launch_inv_t<2, 16, float2>(a, nb, st)));
            else if (mt == KP_C32_BF16) KP_TRY((launch_inv_t<2, 16, __nv_bfloat162>(a, nb, st)));
            else KP_TRY((launch_inv_t<2, 16, __half2>(a, nb, st)));
        } else {
            if (mt == KP_C64) KP_TRY((launch_inv_t<3, 8, float2>(a, nb, st)));
            else if (mt == KP_C32_BF16) KP_TRY((launch_inv_t<3, 8, __nv_bfloat162>(a, nb, st)));
            else KP_TRY((launch_inv_t<3, 8, __half2>(a, nb, st)));
        }
        p->launches += 1;
    }
    return KP_OK;
}

// Level arguments of the prox of one plan (the standalone level kernels' arguments of
// wavelet_prox_levels), forward level lev or inverse level lev; *nb = its blocks.
static LevelArgs prox_level_args(kp_plan p, float lambda, int lev, bool fwd, int* nb) {
    const Geom& g = p->geo;
    const int L = p->P.wavelet_levels;
    const int T = wt_tile(g.D);
    float2* ll[2] = {p->d_wl0, p->d_wl1};
    LevelArgs a{};
    int bdim[MAXD], hdim[MAXD];
    *nb = 1;
    for (int d = 0; d < g.D; ++d) {
        bdim[d] = g.n[d] >> lev;
        hdim[d] = bdim[d] / 2;
        a.b[d] = bdim[d];
        a.tiles[d] = fwd ? (hdim[d] + T - 1) / T : (bdim[d] + 2 * T - 1) / (2 * T);
        *nb *= a.tiles[d];
    }
    a.coef = full_view(p->d_w, g);
    a.lev_last = lev == L - 1;
    a.sched = p->d_sched;
    a.iter = p->d_iter;
    if (fwd) {
        a.src = lev == 0 ? full_view(p->d_z, g) : dense_view(ll[(lev - 1) & 1], bdim, g.D);
        a.dst = dense_view(ll[lev & 1], hdim, g.D);
        a.lambda = lambda;
    } else {
        a.src = dense_view(ll[lev & 1], hdim, g.D);
        a.dst = lev == 0 ? full_view(p->d_x, g) : dense_view(ll[(lev - 1) & 1], bdim, g.D);
        a.lev_first = lev == 0;
        if (lev == 0) {
            a.x = p->d_x;
            a.xbar = p->d_xbar;
            a.fgrid = p->fft3 ? nullptr : p->d_grid;      // the own FFT forms the pre-step itself
            a.maps = p->d_maps;
            a.apod = p->d_apod;
            a.geo = g;
        }
    }
    return a;
}

kp_status batch_wavelet_build(const std::vector<kp_plan>& ps, const std::vector<int>& regs,
                              const std::vector<float>& lams, BatchIter& bi) {
    int Lmax = 0;
    for (size_t i = 0; i < ps.size(); ++i)
        if (regs[i] == KP_REG_L1_WAVELET) Lmax = std::max(Lmax, ps[i]->P.wavelet_levels);
    bi.fwd.resize(Lmax);
    bi.inv.resize(Lmax);
    for (int dir = 0; dir < 2; ++dir)
        for (int lev = 0; lev < Lmax; ++lev) {
            std::vector<LevelArgs> ds;
            std::vector<int> boff(1, 0);
            for (size_t i = 0; i < ps.size(); ++i) {
                if (regs[i] != KP_REG_L1_WAVELET || lev >= ps[i]->P.wavelet_levels) continue;
                int nb = 0;
                ds.push_back(prox_level_args(ps[i], lams[i], lev, dir == 0, &nb));
                boff.push_back(boff.back() + nb);
            }
            KP_TRY(phase_upload(dir == 0 ? bi.fwd[lev] : bi.inv[lev], ds.data(), ds.size() * sizeof(LevelArgs),
                                (int)ds.size(), boff));
        }
    return KP_OK;
}

// Forward levels 0 .. Lmax-1, then inverse levels Lmax-1 .. 0 (2D, tiles of 16).
kp_status batch_wavelet_launch(const BatchIter& bi, cudaStream_t st) {
    constexpr int D = 2, T = 16;
    static PerDeviceOnce attr_f, attr_i[3];
    size_t smf, smi;
    {
        constexpr int EI = 2 * T + 6, E = T + 4;
        smf = ((size_t)EI * EI + (size_t)EI * 2 * T) * sizeof(float2);
        smi = ((size_t)(2 * E) * (2 * E) + (size_t)(2 * E) * 2 * T) * sizeof(float2);
    }
    if (attr_f.first())
        KP_TRY_CUDA(cudaFuncSetAttribute(k_dwt_fwd_level_b<D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    for (size_t lev = 0; lev < bi.fwd.size(); ++lev) {
        const BatchPhase& ph = bi.fwd[lev];
        if (ph.nblocks == 0) continue;
        k_dwt_fwd_level_b<D, T><<<ph.nblocks, 256, smf, st>>>((const LevelArgs*)ph.d_desc, ph.d_boff, ph.ncase);
        KP_LAUNCH_CHECK();
    }
    for (int lev = (int)bi.inv.size() - 1; lev >= 0; --lev) {
        const BatchPhase& ph = bi.inv[lev];
        if (ph.nblocks == 0) continue;
        switch (bi.mt) {
            case KP_C64:
                if (attr_i[0].first())
                    KP_TRY_CUDA(cudaFuncSetAttribute(k_dwt_inv_level_b<D, T, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
                k_dwt_inv_level_b<D, T, float2><<<ph.nblocks, 256, smi, st>>>((const LevelArgs*)ph.d_desc, ph.d_boff, ph.ncase);
                break;
            case KP_C32_BF16:
                if (attr_i[1].first())
                    KP_TRY_CUDA(cudaFuncSetAttribute(k_dwt_inv_level_b<D, T, __nv_bfloat162>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
                k_dwt_inv_level_b<D, T, __nv_bfloat162><<<ph.nblocks, 256, smi, st>>>((const LevelArgs*)ph.d_desc, ph.d_boff, ph.ncase);
                break;
            default:
                if (attr_i[2].first())
                    KP_TRY_CUDA(cudaFuncSetAttribute(k_dwt_inv_level_b<D, T, __half2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
                k_dwt_inv_level_b<D, T, __half2><<<ph.nblocks, 256, smi, st>>>((const LevelArgs*)ph.d_desc, ph.d_boff, ph.ncase);
                break;
        }
        KP_LAUNCH_CHECK();
    }
    return KP_OK;
}

kp_status wavelet_apply(kp_plan p, const float2* in, float2* out, bool forward, cudaStream_t st) {
    if (in == out) {
        // the level kernels read the input while writing the output: stage a copy
        KP_TRY_CUDA(cudaMemcpyAsync(p->d_w, in, p->geo.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
        in = p->d_w;
    }
    if (forward) return wavelet_forward(p, in, out, st);
    return wavelet_inverse(p, in, out, st);
}

}  // namespace kp

namespace kp {

// ================================================================ fused primal step
// One persistent cooperative kernel per PDHG iteration after the inverse FFT (Sec. 4.1):
//   z = x - tau_k A^H u  (coil combine + apodisation of the adjoint grid)
//   l2:  x_new = z / (1 + tau_k lambda)
//   l1:  x_new = W^H S_{tau_k lambda}(W z), level by level with grid barriers in between
//   xbar = x_new + theta_k (x_new - x),  x = x_new,
//   forward pre-step of the next iteration: grid_c = s_c xbar / Phi (image region only),
//   iteration counter += 1.
// Grid barrier: arrival counter + generation word in device memory; every wait is bounded
// (about a second of SM clock), after which the kernel records a timeout in *err and carries
// on (the host reports KP_ETIMEOUT).

// Grid-wide barrier of the persistent kernel: a 64-bit arrival counter that only grows.  Each
// barrier adds exactly gridDim.x, so at the start of every barrier the counter is a multiple
// of gridDim.x; a block's arrival returns the old value, from which it knows the count that
// ends this barrier, and waits until the counter reaches it.  One atomic per block and no
// reset.  The wait is bounded (about one second of clock64); on timeout the block sets *err
// and continues, and the solver reports KP_ETIMEOUT (the counter is cleared before each solve).
struct GridBarrier {
    unsigned long long count;
};

__device__ __forceinline__ void grid_barrier(GridBarrier* b, int* err, long long limit) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned long long old;
        asm volatile("atom.add.relaxed.gpu.global.u64 %0, [%1], 1;" : "=l"(old) : "l"(&b->count) : "memory");
        const unsigned long long target = (old / gridDim.x + 1) * gridDim.x;
        const long long t0 = clock64();
        for (;;) {
            unsigned long long cur;
            asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(cur) : "l"(&b->count) : "memory");
            if (cur >= target) break;
            if (clock64() - t0 > limit) {          // the plan's limit (default about a second)
                atomicExch(err, 1);
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
}

struct PrimalArgs {
    const float2* grid2;   // adjoint grid after the inverse FFT
    const void* maps;
    const float* apod;
    Geom geo;
    float2* x;
    float2* xbar;
    float2* z;
    float2* coef;          // wavelet coefficients
    float2* ll0;
    float2* ll1;
    float2* fgrid;         // forward grid of the next iteration (image region written)
    const float* sched;
    int* iter;
    float lambda;
    int levels;
    float2* grid2w;        // the same grid, written: split spreading tiles cleared once read
    const int* split;
    int n_split;
    Tiles tiles;
    GridBarrier* bar;
    int* err;
    long long wait;        // limit of each grid-barrier wait (SM clock cycles)
};

template <int D, int T>
__device__ __forceinline__ LevelArgs level_args(const PrimalArgs& a, int lev, bool fwd, int k) {
    LevelArgs la{};
    const Geom& g = a.geo;
    int bdim[MAXD], hdim[MAXD];
    int nb = 1;
    for (int d = 0; d < D; ++d) {
        bdim[d] = g.n[d] >> lev;
        hdim[d] = bdim[d] / 2;
        la.b[d] = bdim[d];
        la.tiles[d] = fwd ? (hdim[d] + T - 1) / T : (bdim[d] + 2 * T - 1) / (2 * T);
        nb *= la.tiles[d];
    }
    la.tiles_total = nb;
    auto full = [&](float2* p) { View v{}; v.p = p; int64_t s = 1; for (int d = D - 1; d >= 0; --d) { v.s[d] = s; s *= g.n[d]; } return v; };
    auto dense = [&](float2* p, const int* dims) { View v{}; v.p = p; int64_t s = 1; for (int d = D - 1; d >= 0; --d) { v.s[d] = s; s *= dims[d]; } return v; };
    float2* ll[2] = {a.ll0, a.ll1};
    la.coef = full(a.coef);
    la.lev_last = lev == a.levels - 1;
    la.sched = a.sched;
    la.iter = a.iter;
    la.lambda = a.lambda;
    la.geo = g;
    if (fwd) {
        la.src = lev == 0 ? full(a.z) : dense(ll[(lev - 1) & 1], bdim);
        la.dst = dense(ll[lev & 1], hdim);
    } else {
        la.src = dense(ll[lev & 1], hdim);
        la.dst = lev == 0 ? full(a.x) : dense(ll[(lev - 1) & 1], bdim);
        la.lev_first = lev == 0;
        la.x = lev == 0 ? a.x : nullptr;
        la.xbar = lev == 0 ? a.xbar : nullptr;
        la.fgrid = lev == 0 ? a.fgrid : nullptr;
        la.maps = a.maps;
        la.apod = a.apod;
    }
    (void)k;
    return la;
}

constexpr int PF_THREADS = 1024;

// Clears the split spreading tiles' regions of grid2 (all coils), CTA-strided over tiles, so
// the next spread can accumulate into them without a separate clearing kernel.
template <int D>
__device__ void zero_split_tiles(const PrimalArgs& a) {
    const Geom& g = a.geo;
    const Tiles& tl = a.tiles;
    int P = 1;
    for (int d = 0; d < D; ++d) P *= tl.ts[d];
    for (int t = blockIdx.x; t < a.n_split; t += gridDim.x) {
        int r = a.split[t], o[MAXD], e[MAXD];
        for (int d = D - 1; d >= 0; --d) {
            const int tc = r % tl.nt[d];
            r /= tl.nt[d];
            o[d] = tc * tl.ts[d];
            e[d] = min(tl.ts[d], g.g[d] - o[d]);
        }
        for (int i = threadIdx.x; i < g.C * P; i += blockDim.x) {
            const int c = i / P;
            int rr = i - c * P, lidx[MAXD];
            for (int d = D - 1; d >= 0; --d) { lidx[d] = rr % tl.ts[d]; rr /= tl.ts[d]; }
            bool in = true;
            int64_t gflat = 0;
            for (int d = 0; d < D; ++d) {
                if (lidx[d] >= e[d]) in = false;
                gflat = gflat * g.g[d] + tunshift(o[d] + lidx[d], tl.sh[d], g.g[d]);
            }
            if (in && KP_INB(13, gflat, g.G)) a.grid2w[(size_t)c * g.G + gflat] = make_float2(0.f, 0.f);
        }
    }
}

template <int D, int T, typename MT, int REG>
__global__ void __launch_bounds__(PF_THREADS, 1) k_primal_fused(PrimalArgs a) {
    extern __shared__ float2 sm[];
    const Geom& g = a.geo;
    const int k = *a.iter;
    const float tau = a.sched[3 * k + 1], theta = a.sched[3 * k + 2];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < g.N; j += stride) {
        const float2 ah = adj_pixel<D, MT>(a.grid2, (const MT*)a.maps, a.apod, g, j);
        const float2 xo = a.x[j];
        const float2 zz = make_float2(xo.x - tau * ah.x, xo.y - tau * ah.y);
        if (REG == 0) {
            const float sc = 1.f / (1.f + tau * a.lambda);
            const float2 xn = make_float2(zz.x * sc, zz.y * sc);
            const float2 xb = make_float2(xn.x + theta * (xn.x - xo.x), xn.y + theta * (xn.y - xo.y));
            a.x[j] = xn;
            a.xbar[j] = xb;
            if (a.fgrid) pre_pixel<D, MT>(a.fgrid, (const MT*)a.maps, a.apod, g, j, xb);
        } else {
            a.z[j] = zz;
        }
    }
    if (REG == 1) {
        grid_barrier(a.bar, a.err, a.wait);
        zero_split_tiles<D>(a);   // grid2 has been read by every block
        for (int lev = 0; lev < a.levels; ++lev) {
            const LevelArgs la = level_args<D, T>(a, lev, true, k);
            for (int t = blockIdx.x; t < la.tiles_total; t += gridDim.x) fwd_level_tile<D, T>(la, t, sm);
            grid_barrier(a.bar, a.err, a.wait);
        }
        for (int lev = a.levels - 1; lev >= 0; --lev) {
            const LevelArgs la = level_args<D, T>(a, lev, false, k);
            for (int t = blockIdx.x; t < la.tiles_total; t += gridDim.x) inv_level_tile<D, T, MT>(la, t, sm);
            if (lev > 0) grid_barrier(a.bar, a.err, a.wait);
        }
    }
    grid_barrier(a.bar, a.err, a.wait);   // every block has read the iteration counter (and grid2)
    if (REG == 0) zero_split_tiles<D>(a);
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.iter = k + 1;
}

template <int D, int T>
static size_t primal_smem() {
    constexpr int EI = 2 * T + 6, E = T + 4;
    size_t f = 1, f1 = 1, v = 1, v1 = 1;
    for (int d = 0; d < D; ++d) {
        f *= EI; f1 *= (d == D - 1 ? 2 * T : EI);
        v *= 2 * E; v1 *= (d == D - 1 ? 2 * T : 2 * E);
    }
    return std::max(f + f1, v + v1) * sizeof(float2);
}

template <int D, int T, typename MT, int REG>
static kp_status launch_primal(kp_plan p, const PrimalArgs& a, cudaStream_t st) {
    auto kern = k_primal_fused<D, T, MT, REG>;
    const size_t smem = REG == 1 ? primal_smem<D, T>() : 0;
    static std::atomic<int> blocks_cache[64];   // per device: CTAs of the cooperative grid
    int dev = 0;
    KP_TRY_CUDA(cudaGetDevice(&dev));
    int nblk = blocks_cache[dev & 63].load();
    if (nblk == 0) {
        KP_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
        int sms = 0, per = 0;
        KP_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        KP_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, PF_THREADS, smem));
        if (per < 1) { set_error("fused primal kernel does not fit on an SM"); return KP_EINTERNAL; }
        nblk = sms;   // one CTA per SM: the barrier's arrival count stays small
        blocks_cache[dev & 63].store(nblk);
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)nblk);
    cfg.blockDim = dim3(PF_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    KP_TRY_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
    p->launches += 1;
    return KP_OK;
}


// ---------------------------------------------------------------- l1 prox by one cluster (2D)
// The l1-wavelet prox W^H S_t(W z) of a 2D image, with the extrapolation, by one cluster of
// NC = 16 or 8 CTAs (one per SM, 1024 threads) instead of tiled passes separated by grid-wide barriers.
// CTA r holds image rows [r R0, (r + 1) R0) (R0 = n0 / NC) in shared memory and transforms
// them in place in a Mallat layout local to its row block: at level l its block is the top-left
// (R0 >> l) x (n1 >> l) corner; the x pass (along rows) is local, the y pass reads the rows it
// needs from the CTAs that own them through distributed shared memory (rows of a level are
// owned by CTA row / (R0 >> l)), and the CTAs meet at hardware cluster barriers.  Forward
// levels: x pass into T, cluster barrier, y pass from T into the block (details and, at the
// last level, the approximation soft-thresholded).  Inverse levels: y pass reading the owners'
// coefficient rows into T, cluster barrier, x pass into the block, cluster barrier.  The
// coefficients are the same as those of the tiled transform (same filters, periodic indexing),
// only stored in a different order, so the prox is the same up to rounding order.
namespace cgc = cooperative_groups;

constexpr int CP_THREADS = 1024;

__device__ __forceinline__ int cp_wrap(int i, int len) {
    while (i >= len) i -= len;
    while (i < 0) i += len;
    return i;
}

template <int NC>
__global__ void __launch_bounds__(CP_THREADS)
k_wprox_cluster(const float2* __restrict__ z, float2* __restrict__ x, float2* __restrict__ xbar,
                const float* __restrict__ sched, const int* __restrict__ iter, float lambda, int n0, int n1, int L) {
    cgc::cluster_group cl = cgc::this_cluster();
    const int r = (int)cl.block_rank();
    extern __shared__ __align__(16) float2 smc[];
    const int R0 = n0 / NC;
    float2* A = smc;                        // [R0][n1], row stride n1 at every level
    float2* T0 = A + (size_t)R0 * n1;       // [R0][n1] dense per level (even levels, inverse)
    float2* T1 = T0 + (size_t)R0 * n1;      // [R0/2][n1/2] dense (odd forward levels)
    const int k = *iter;
    const float thr = sched[3 * k + 1] * lambda, theta = sched[3 * k + 2];
    const int tid = threadIdx.x, nt = blockDim.x;
    const size_t row0 = (size_t)r * R0 * n1;
    for (int i = tid; i < R0 * n1; i += nt) A[i] = z[row0 + i];
    __syncthreads();
    float hh[8], gg[8];
#pragma unroll
    for (int n = 0; n < 8; ++n) { hh[n] = c_wh[n]; gg[n] = c_wg[n]; }
    for (int lev = 0; lev < L; ++lev) {
        const int Rl = R0 >> lev, cw = n1 >> lev, nl = n0 >> lev, half = cw / 2, R1 = Rl / 2;
        float2* T = (lev & 1) ? T1 : T0;
        // x pass (local): thread per (row, k); a[k] and d[k] from the same 8 inputs
        for (int o = tid; o < Rl * half; o += nt) {
            const int i = o / half, kq = o - i * half;
            const float2* row = A + (size_t)i * n1;
            int idx = 2 * kq;
            float2 a = make_float2(0.f, 0.f), d = a;
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const float2 v = row[idx];
                a.x = fmaf(hh[n], v.x, a.x); a.y = fmaf(hh[n], v.y, a.y);
                d.x = fmaf(gg[n], v.x, d.x); d.y = fmaf(gg[n], v.y, d.y);
                if (++idx == cw) idx = 0;
            }
            T[(size_t)i * cw + kq] = a;
            T[(size_t)i * cw + half + kq] = d;
        }
        cl.sync();
        // y pass: thread per (k, column); rows 2k .. 2k + 7 from their owners
        for (int o = tid; o < R1 * cw; o += nt) {
            const int kk = o / cw, c = o - kk * cw;
            // row 2k + n (periodic) lives in CTA own at local row lr; the level's nl rows are
            // exactly NC blocks of Rl, so (own, lr) step and wrap together
            const int row = cp_wrap(2 * (r * R1 + kk), nl);
            int own = row / Rl, lr = row - own * Rl;
            const float2* Tr = cl.map_shared_rank(T, own);
            float2 a = make_float2(0.f, 0.f), d = a;
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const float2 v = Tr[(size_t)lr * cw + c];
                a.x = fmaf(hh[n], v.x, a.x); a.y = fmaf(hh[n], v.y, a.y);
                d.x = fmaf(gg[n], v.x, d.x); d.y = fmaf(gg[n], v.y, d.y);
                if (++lr == Rl) {
                    lr = 0;
                    if (++own == NC) own = 0;
                    Tr = cl.map_shared_rank(T, own);
                }
            }
            if (c >= half || lev == L - 1) a = soft(a, thr);   // the approximation stays for the next level
            A[(size_t)kk * n1 + c] = a;
            A[(size_t)(R1 + kk) * n1 + c] = soft(d, thr);
        }
        __syncthreads();
    }
    cl.sync();
    for (int lev = L - 1; lev >= 0; --lev) {
        const int Rl = R0 >> lev, cw = n1 >> lev, half = cw / 2, R1 = Rl / 2;
        // y pass: thread per (output row pair, column): rows 2m and 2m + 1 from coefficient
        // rows m - 3 .. m (periodic) of the owners
        for (int o = tid; o < R1 * cw; o += nt) {
            const int mm = o / cw, c = o - mm * cw;
            // coefficient row mg - t (periodic over nh = NC R1 rows) lives in CTA own at local
            // row lk; stepping down, (own, lk) wrap together
            int own = r, lk = mm;
            const float2* Ar = cl.map_shared_rank(A, own);
            float2 e = make_float2(0.f, 0.f), od = e;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (t > 0 && --lk < 0) {
                    lk = R1 - 1;
                    if (--own < 0) own = NC - 1;
                    Ar = cl.map_shared_rank(A, own);
                }
                const float2 av = Ar[(size_t)lk * n1 + c], dv = Ar[(size_t)(R1 + lk) * n1 + c];
                // x[2 mg] uses n = 2t, x[2 mg + 1] uses n = 2t + 1, both at k = mg - t
                e.x = fmaf(hh[2 * t], av.x, fmaf(gg[2 * t], dv.x, e.x));
                e.y = fmaf(hh[2 * t], av.y, fmaf(gg[2 * t], dv.y, e.y));
                od.x = fmaf(hh[2 * t + 1], av.x, fmaf(gg[2 * t + 1], dv.x, od.x));
                od.y = fmaf(hh[2 * t + 1], av.y, fmaf(gg[2 * t + 1], dv.y, od.y));
            }
            T0[(size_t)(2 * mm) * cw + c] = e;
            T0[(size_t)(2 * mm + 1) * cw + c] = od;
        }
        cl.sync();                                             // every owner's rows have been read
        // x pass (local): thread per (row, output pair)
        for (int o = tid; o < Rl * half; o += nt) {
            const int jj = o / half, mq = o - jj * half;
            const float2* t = T0 + (size_t)jj * cw;
            float2 e = make_float2(0.f, 0.f), od = e;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int kq = cp_wrap(mq - u, half);
                const float2 av = t[kq], dv = t[half + kq];
                e.x = fmaf(hh[2 * u], av.x, fmaf(gg[2 * u], dv.x, e.x));
                e.y = fmaf(hh[2 * u], av.y, fmaf(gg[2 * u], dv.y, e.y));
                od.x = fmaf(hh[2 * u + 1], av.x, fmaf(gg[2 * u + 1], dv.x, od.x));
                od.y = fmaf(hh[2 * u + 1], av.y, fmaf(gg[2 * u + 1], dv.y, od.y));
            }
            A[(size_t)jj * n1 + 2 * mq] = e;
            A[(size_t)jj * n1 + 2 * mq + 1] = od;
        }
        cl.sync();                                             // the next level reads these rows
    }
    for (int i = tid; i < R0 * n1; i += nt) {                 // extrapolation (Sec. 4.1)
        const float2 xn = A[i], xo = x[row0 + i];
        xbar[row0 + i] = make_float2(xn.x + theta * (xn.x - xo.x), xn.y + theta * (xn.y - xo.y));
        x[row0 + i] = xn;
    }
}

// After the cluster prox: blocks below nb_pre write the next iteration's coil multiply /
// apodise / pad of xbar into the image region of the forward grid (the zero padding stays from
// solve set-up); block nb_pre + t clears split spreading tile t of the adjoint grid; block 0
// advances the iteration counter.  32-bit index arithmetic (2D).
template <typename MT>
__global__ void __launch_bounds__(256)
k_pre_clear(const float2* __restrict__ xbar, const MT* __restrict__ maps, const float* __restrict__ apod, Geom geo,
            float2* __restrict__ fgrid, int nb_pre, const int* __restrict__ split, Tiles tl, float2* __restrict__ grid2,
            int* __restrict__ iter) {
    const int n0 = geo.n[0], n1 = geo.n[1], g0 = geo.g[0], g1 = geo.g[1];
    if ((int)blockIdx.x < nb_pre) {
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n0 * n1; j += nb_pre * blockDim.x) {
            const int iy = j / n1, ix = j - iy * n1;
            const int ny = iy - n0 / 2, nx = ix - n1 / 2;
            const int gy = ny < 0 ? ny + g0 : ny, gx = nx < 0 ? nx + g1 : nx;
            const float a = apod[iy] * apod[n0 + ix];
            float2 v = xbar[j];
            v.x *= a;
            v.y *= a;
            const size_t gi = (size_t)gy * g1 + gx;
            for (int c = 0; c < geo.C; ++c) {
                const float2 sv = ldc<MT>(maps, (size_t)c * geo.N + j);
                fgrid[(size_t)c * geo.G + gi] = cmul(sv, v);
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) *iter += 1;
        return;
    }
    int t = split[blockIdx.x - nb_pre];
    const int tc1 = t % tl.nt[1], tc0 = t / tl.nt[1];
    const int o0 = tc0 * tl.ts[0], o1 = tc1 * tl.ts[1];
    const int e0 = min(tl.ts[0], g0 - o0), e1 = min(tl.ts[1], g1 - o1);
    for (int i = threadIdx.x; i < geo.C * e0 * e1; i += blockDim.x) {
        const int c = i / (e0 * e1), p = i - c * e0 * e1;
        const int l0 = p / e1, l1 = p - l0 * e1;
        const size_t gflat = (size_t)tunshift(o0 + l0, tl.sh[0], g0) * g1 + tunshift(o1 + l1, tl.sh[1], g1);
        grid2[(size_t)c * geo.G + gflat] = make_float2(0.f, 0.f);
    }
}

static size_t cluster_smem(const Geom& g, int nc) {
    const size_t R0 = (size_t)g.n[0] / nc, n1 = (size_t)g.n[1];
    return (2 * R0 * n1 + (R0 / 2) * (n1 / 2)) * sizeof(float2);
}

template <int NC>
static cudaLaunchConfig_t cluster_cfg(size_t sm, cudaStream_t st, cudaLaunchAttribute* at) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(NC);
    cfg.blockDim = dim3(CP_THREADS);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = NC;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

// Sets the kernel's attributes on the current device and asks whether one cluster fits.
template <int NC>
static SmemLimit& cluster_limit() {
    static SmemLimit lim;
    return lim;
}

template <int NC>
static bool cluster_fits(size_t sm) {
    if (cluster_limit<NC>().ensure(k_wprox_cluster<NC>, sm) != cudaSuccess ||
        (NC > 8 && cudaFuncSetAttribute(k_wprox_cluster<NC>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cluster_cfg<NC>(sm, nullptr, at);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_wprox_cluster<NC>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclusters >= 1;
}

// Whether the 2D l1 prox can run as one cluster of 16 (else 8) CTAs: rows split evenly over
// the CTAs with every level's row block even, shared memory within 200 KB, and the device able
// to place the cluster.  The choice is made at solve set-up (outside any graph capture).  The
// environment variable KPDHG_NO_CLUSTER_PROX=1 keeps the cooperative kernel.
bool cluster_prox_ok(kp_plan p) {
    if (p->cluster_prox >= 0) return p->cluster_prox > 0;
    const Geom& g = p->geo;
    const int L = p->P.wavelet_levels;
    int chosen = 0;
    bool allowed = g.D == 2 && L >= 1;
    if (const char* ev = getenv("KPDHG_NO_CLUSTER_PROX"))
        if (atoi(ev) != 0) allowed = false;
    for (int nc : {16, 8}) {
        if (!allowed || chosen) break;
        if (g.n[0] % nc != 0 || ((g.n[0] / nc) % (1 << L)) != 0) continue;
        const size_t sm = cluster_smem(g, nc);
        if (sm > 200 * 1024) continue;
        if (nc == 16 ? cluster_fits<16>(sm) : cluster_fits<8>(sm)) chosen = nc;
    }
    p->cluster_prox = chosen;
    return chosen > 0;
}

// One PDHG primal step for a 2D l1 plan on the cluster path: adjoint combine into z, the
// cluster prox and extrapolation, then the pre-step, split-tile clearing and counter.
kp_status primal_cluster(kp_plan p, float lambda, cudaStream_t st) {
    const Geom& g = p->geo;
    const int nc = p->cluster_prox;
    KP_TRY(adjoint_primal(p, KP_REG_L1_WAVELET, lambda, st));
    mark(p, PH_DWT_FWD, st);
    const size_t sm = cluster_smem(g, nc);
    cudaLaunchAttribute at[1];
    if (nc == 16) {
        KP_TRY_CUDA(cluster_limit<16>().ensure(k_wprox_cluster<16>, sm));
        cudaLaunchConfig_t cfg = cluster_cfg<16>(sm, st, at);
        KP_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_wprox_cluster<16>, (const float2*)p->d_z, p->d_x, p->d_xbar,
                                       (const float*)p->d_sched, (const int*)p->d_iter, lambda, g.n[0], g.n[1],
                                       p->P.wavelet_levels));
    } else {
        KP_TRY_CUDA(cluster_limit<8>().ensure(k_wprox_cluster<8>, sm));
        cudaLaunchConfig_t cfg = cluster_cfg<8>(sm, st, at);
        KP_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_wprox_cluster<8>, (const float2*)p->d_z, p->d_x, p->d_xbar,
                                       (const float*)p->d_sched, (const int*)p->d_iter, lambda, g.n[0], g.n[1],
                                       p->P.wavelet_levels));
    }
    p->launches += 1;
    mark(p, PH_FWD_PRE, st);
    const int nb_pre = 2 * 152;
    const unsigned nb = (unsigned)(nb_pre + (p->spread_variant >= 10 ? 0 : p->n_split));   // 10-12 store every point
    const kp_cdtype mt = p->maps_t;
    if (mt == KP_C64)
        k_pre_clear<float2><<<nb, 256, 0, st>>>(p->d_xbar, (const float2*)p->d_maps, p->d_apod, g, p->d_grid, nb_pre,
                                                p->d_split, p->tiles, p->d_grid2, p->d_iter);
    else if (mt == KP_C32_BF16)
        k_pre_clear<__nv_bfloat162><<<nb, 256, 0, st>>>(p->d_xbar, (const __nv_bfloat162*)p->d_maps, p->d_apod, g, p->d_grid,
                                                        nb_pre, p->d_split, p->tiles, p->d_grid2, p->d_iter);
    else
        k_pre_clear<__half2><<<nb, 256, 0, st>>>(p->d_xbar, (const __half2*)p->d_maps, p->d_apod, g, p->d_grid, nb_pre,
                                                 p->d_split, p->tiles, p->d_grid2, p->d_iter);
    KP_LAUNCH_CHECK();
    p->launches += 1;
    return KP_OK;
}

kp_status primal_fused(kp_plan p, int reg, float lambda, cudaStream_t st) {
    const Geom& g = p->geo;
    PrimalArgs a{};
    a.grid2 = p->d_grid2;
    a.maps = p->d_maps;
    a.apod = p->d_apod;
    a.geo = g;
    a.x = p->d_x;
    a.xbar = p->d_xbar;
    a.z = p->d_z;
    a.coef = p->d_w;
    a.ll0 = p->d_wl0;
    a.ll1 = p->d_wl1;
    a.fgrid = p->fft3 ? nullptr : p->d_grid;            // the own FFT forms the pre-step itself
    a.sched = p->d_sched;
    a.iter = p->d_iter;
    a.lambda = lambda;
    a.levels = p->P.wavelet_levels;
    a.grid2w = p->d_grid2;
    a.split = p->d_split;
    a.n_split = p->spread_variant >= 10 ? 0 : (int)p->n_split;   // two-phase spreading stores every point
    a.tiles = p->tiles;
    a.bar = (GridBarrier*)p->d_bar;
    a.err = p->d_flag + KP_FLAG_TIMEOUT;
    a.wait = p->wait_cycles;
    mark(p, PH_ADJ, st);
    const kp_cdtype mt = p->maps_t;
#define KP_PRIMAL(DD, TT)                                                                          \
    do {                                                                                           \
        if (reg == KP_REG_L2) {                                                                    \
            if (mt == KP_C64) return launch_primal<DD, TT, float2, 0>(p, a, st);                   \
            if (mt == KP_C32_BF16) return launch_primal<DD, TT, __nv_bfloat162, 0>(p, a, st);      \
            return launch_primal<DD, TT, __half2, 0>(p, a, st);                                    \
        }                                                                                          \
        if (mt == KP_C64) return launch_primal<DD, TT, float2, 1>(p, a, st);                       \
        if (mt == KP_C32_BF16) return launch_primal<DD, TT, __nv_bfloat162, 1>(p, a, st);          \
        return launch_primal<DD, TT, __half2, 1>(p, a, st);                                        \
    } while (0)
    if (g.D == 2) KP_PRIMAL(2, 16);
    KP_PRIMAL(3, 8);
#undef KP_PRIMAL
}

}  // namespace kp
