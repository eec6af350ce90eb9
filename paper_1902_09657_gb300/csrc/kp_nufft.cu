// Multi-coil SENSE NUFFT pair A = F_nu S and A^H on sm_103a (Sec. 2 Eq. model_i;
// Sec. 6: Kaiser-Bessel gridding following Beatty et al., oversampling g/n, width 4).
//
// Forward:  fwd_pre (coil multiply, 1/Phi apodisation, centred zero padding; writes the
//           whole grid) -> cuFFT C2C forward, batch C -> interp (W^D taps per sample,
//           one thread per sorted sample, all coils, N^{-1/2}).
// Adjoint:  spread (one CTA per (tile, chunk) work item; a warp takes one sample at a
//           time with its lanes over (tap, coil) pairs, so shared-memory atomics within a
//           warp never collide; single-chunk tiles store straight to the grid, split tiles
//           store partial tiles that a reduction pass sums) -> cuFFT C2C inverse ->
//           adj_post (crop, 1/Phi, conj(s_c) coil combine, N^{-1/2}).
// The grid coordinates t = f g/n are float32; the first tap is k0 = ceil(t) - W/2, which equals
// ceil(t - W/2) exactly and involves no rounding, so |t - k| <= W/2 for every tap.
#include "kp_internal.cuh"

namespace kp {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ int wrapg(int k, int g) { return k < 0 ? k + g : (k >= g ? k - g : k); }

// Kaiser-Bessel window of width 4: I0(beta sqrt(1 - (u/2)^2)) on |u| <= 2.
__device__ __forceinline__ float kbw(float u, float beta) {
    float h = 0.5f * u;
    float a = 1.f - h * h;
    return a >= 0.f ? cyl_bessel_i0f(beta * sqrtf(a)) : 0.f;
}

template <int D>
struct Taps {
    int off[D][KW];     // grid offset contribution of tap j on axis d (already times the axis stride)
    int idx[D][KW];     // wrapped grid index on axis d
    float w[D][KW];
};

template <int D>
__device__ __forceinline__ void make_taps(const float* __restrict__ t, int64_t s, const Geom& geo, Taps<D>& tp) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
        float td = t[(int64_t)d * geo.M + s];
        int k0 = (int)ceilf(td) - KW / 2;
        int stride = 1;
        for (int e = d + 1; e < D; ++e) stride *= geo.g[e];
#pragma unroll
        for (int j = 0; j < KW; ++j) {
            int k = k0 + j;
            tp.w[d][j] = kbw(td - (float)k, geo.beta[d]);
            int ix = wrapg(k, geo.g[d]);
            tp.idx[d][j] = ix;
            tp.off[d][j] = ix * stride;
        }
    }
}

// sum over taps of w * grid[c] for one coil.
template <int D>
__device__ __forceinline__ float2 gather_coil(const float2* __restrict__ base, const Taps<D>& tp) {
    float2 acc = make_float2(0.f, 0.f);
    if (D == 2) {
#pragma unroll
        for (int a = 0; a < KW; ++a) {
#pragma unroll
            for (int b = 0; b < KW; ++b) {
                float w = tp.w[0][a] * tp.w[1][b];
                float2 v = __ldg(base + tp.off[0][a] + tp.off[D - 1][b]);
                acc.x = fmaf(w, v.x, acc.x);
                acc.y = fmaf(w, v.y, acc.y);
            }
        }
    } else {
#pragma unroll
        for (int a = 0; a < KW; ++a) {
#pragma unroll
            for (int b = 0; b < KW; ++b) {
                float wab = tp.w[0][a] * tp.w[1 % D][b];
                int oab = tp.off[0][a] + tp.off[1 % D][b];
#pragma unroll
                for (int c = 0; c < KW; ++c) {
                    float w = wab * tp.w[D - 1][c];
                    float2 v = __ldg(base + oab + tp.off[D - 1][c]);
                    acc.x = fmaf(w, v.x, acc.x);
                    acc.y = fmaf(w, v.y, acc.y);
                }
            }
        }
    }
    return acc;
}

// ---------------------------------------------------------------- forward: pre
// Pixel index (row-major, centred) for grid index i on axis d, or -1 outside the image.
__device__ __forceinline__ int pix_of_grid(int i, int n, int g) {
    int h = n / 2;
    if (i < n - h) return i + h;
    if (i >= g - h) return i - g + h;
    return -1;
}

template <int D, typename MT>
__global__ void k_fwd_pre(const float2* __restrict__ x, const MT* __restrict__ maps, const float* __restrict__ apod,
                          Geom geo, float2* __restrict__ grid) {
    int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= geo.G) return;
    int ii[D];
    int64_t r = gi;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) { ii[d] = (int)(r % geo.g[d]); r /= geo.g[d]; }
    int64_t j = 0;
    float a = 1.f;
    bool inside = true;
    int ao = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        int jd = pix_of_grid(ii[d], geo.n[d], geo.g[d]);
        if (jd < 0) inside = false;
        else a *= apod[ao + jd];
        j = j * geo.n[d] + (jd < 0 ? 0 : jd);
        ao += geo.n[d];
    }
    if (!inside) {
        for (int c = 0; c < geo.C; ++c) grid[(size_t)c * geo.G + gi] = make_float2(0.f, 0.f);
        return;
    }
    float2 xv = x[j];
    xv.x *= a;
    xv.y *= a;
    for (int c = 0; c < geo.C; ++c) {
        float2 s = maps ? ldc<MT>(maps, (size_t)c * geo.N + j) : make_float2(1.f, 0.f);
        grid[(size_t)c * geo.G + gi] = cmul(s, xv);
    }
}

// ---------------------------------------------------------------- forward: interp variants
template <int D, typename OT>
__global__ void k_interp_out(const float* __restrict__ t, const float2* __restrict__ grid, Geom geo,
                             const int* __restrict__ perm, OT* __restrict__ out) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= geo.M) return;
    Taps<D> tp;
    make_taps<D>(t, s, geo, tp);
    int64_t o = perm ? perm[s] : s;
    for (int c = 0; c < geo.C; ++c) {
        float2 v = gather_coil<D>(grid + (size_t)c * geo.G, tp);
        v.x *= geo.rsqrtN;
        v.y *= geo.rsqrtN;
        stc<OT>(out, (size_t)c * geo.M + o, v);
    }
}

template <int D>
__global__ void k_interp_scaled(const float* __restrict__ t, const float2* __restrict__ grid, Geom geo,
                                const float* __restrict__ ps, float2* __restrict__ out) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= geo.M) return;
    Taps<D> tp;
    make_taps<D>(t, s, geo, tp);
    for (int c = 0; c < geo.C; ++c) {
        size_t o = (size_t)c * geo.M + s;
        float2 v = gather_coil<D>(grid + (size_t)c * geo.G, tp);
        float sc = geo.rsqrtN * (ps ? ps[o] : 1.f);
        out[o] = make_float2(v.x * sc, v.y * sc);
    }
}

// PDHG dual step (Sec. 4.1): u <- (u + sigma p (A xbar - y)) / (1 + sigma p).
template <int D, typename YT>
__global__ void k_interp_dual(const float* __restrict__ t, const float2* __restrict__ grid, Geom geo,
                              const YT* __restrict__ ys, const float* __restrict__ ps, float2* __restrict__ u,
                              const float* __restrict__ sched, const int* __restrict__ iter) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= geo.M) return;
    const float sigma = sched[3 * (*iter)];
    Taps<D> tp;
    make_taps<D>(t, s, geo, tp);
    for (int c = 0; c < geo.C; ++c) {
        size_t o = (size_t)c * geo.M + s;
        float2 v = gather_coil<D>(grid + (size_t)c * geo.G, tp);
        float2 y = ldc<YT>(ys, o);
        float sp = sigma * ps[o];
        float inv = 1.f / (1.f + sp);
        float2 uo = u[o];
        float2 un;
        un.x = (uo.x + sp * (v.x * geo.rsqrtN - y.x)) * inv;
        un.y = (uo.y + sp * (v.y * geo.rsqrtN - y.y)) * inv;
        u[o] = un;
    }
}

// ---------------------------------------------------------------- adjoint: spread
constexpr int SP_CH = 16;          // coils per shared-memory pass
constexpr int SP_THREADS = 256;

struct SpreadLayout {
    int ls[MAXD];      // shared-memory strides of the local tile index (padded against bank conflicts)
    int plane;         // floats per coil plane (re and im planes are separate)
    int P;             // unpadded tile points
};

static SpreadLayout spread_layout(const Tiles& tl, int D) {
    SpreadLayout L{};
    int last = D - 1;
    L.ls[last] = 1;
    int ext = tl.ts[last] + 4;
    for (int d = last - 1; d >= 0; --d) {
        L.ls[d] = ext;
        ext *= tl.ts[d] + (d > 0 ? 1 : 0);
    }
    int pl = ext;
    pl = ((pl + 31) / 32) * 32 + 16;
    L.plane = pl;
    L.P = 1;
    for (int d = 0; d < D; ++d) L.P *= tl.ts[d];
    return L;
}

// Weight and shared-memory offset of tap q (axis-major digits, last axis fastest) of a
// sample, or false if that tap falls outside the tile.
template <int D>
__device__ __forceinline__ bool tap_local(int q, const int* k0, const float* td, const int* o, const int* e,
                                          const Geom& geo, const SpreadLayout& L, float& w, int& lo) {
    w = 1.f;
    lo = 0;
    bool ok = true;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) {
        int j = q % KW;
        q /= KW;
        int k = k0[d] + j;
        int l = wrapg(k, geo.g[d]) - o[d];
        if (l < 0 || l >= e[d]) ok = false;
        w *= kbw(td[d] - (float)k, geo.beta[d]);
        lo += l * L.ls[d];
    }
    return ok;
}

template <int D, typename UT>
__global__ void __launch_bounds__(SP_THREADS)
k_spread(const float* __restrict__ t, const UT* __restrict__ u, const int* __restrict__ perm,
         const int* __restrict__ ext, const int4* __restrict__ items, Geom geo, Tiles tl, SpreadLayout L,
         float2* __restrict__ grid, float2* __restrict__ partial) {
    extern __shared__ float sacc[];   // [CH][2][plane]
    const int4 it = items[blockIdx.x];
    const int tile = it.x, beg = it.y, end = it.z, slot = it.w;
    int o[MAXD], e[MAXD];
    {
        int r = tile;
        for (int d = D - 1; d >= 0; --d) {
            int tc = r % tl.nt[d];
            r /= tl.nt[d];
            o[d] = tc * tl.ts[d];
            e[d] = min(tl.ts[d], geo.g[d] - o[d]);
        }
    }
    constexpr int TAPS = D == 2 ? KW * KW : KW * KW * KW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c0 = 0; c0 < geo.C; c0 += SP_CH) {
        const int cc = min(SP_CH, geo.C - c0);
        for (int i = threadIdx.x; i < cc * 2 * L.plane; i += blockDim.x) sacc[i] = 0.f;
        __syncthreads();
        for (int ei = beg + warp; ei < end; ei += nw) {
            const int s = ext[ei];
            const int64_t un = perm ? perm[s] : s;
            // per-axis tap positions relative to the tile, and weights
            float td[D];
            int k0[D];
#pragma unroll
            for (int d = 0; d < D; ++d) {
                td[d] = t[(int64_t)d * geo.M + s];
                k0[d] = (int)ceilf(td[d]) - KW / 2;
            }
            if (TAPS < 32) {
                // 2D: two lanes per tap, each taking every other coil
                constexpr int LPT = TAPS < 32 ? 32 / TAPS : 1;
                const int q = lane % TAPS;
                float w;
                int lo;
                if (tap_local<D>(q, k0, td, o, e, geo, L, w, lo)) {
                    for (int c = lane / TAPS; c < cc; c += LPT) {
                        float2 uv = ldc<UT>(u, (size_t)(c0 + c) * geo.M + un);
                        float* pl = sacc + (size_t)c * 2 * L.plane;
                        atomicAdd(pl + lo, w * uv.x);
                        atomicAdd(pl + L.plane + lo, w * uv.y);
                    }
                }
            } else {
                for (int q = lane; q < TAPS; q += 32) {
                    float w;
                    int lo;
                    if (!tap_local<D>(q, k0, td, o, e, geo, L, w, lo)) continue;
                    for (int c = 0; c < cc; ++c) {
                        float2 uv = ldc<UT>(u, (size_t)(c0 + c) * geo.M + un);
                        float* pl = sacc + (size_t)c * 2 * L.plane;
                        atomicAdd(pl + lo, w * uv.x);
                        atomicAdd(pl + L.plane + lo, w * uv.y);
                    }
                }
            }
        }
        __syncthreads();
        // write out the tile (or its partial)
        for (int i = threadIdx.x; i < cc * L.P; i += blockDim.x) {
            const int c = i / L.P;
            int r = i % L.P;
            int lidx[MAXD];
            for (int d = D - 1; d >= 0; --d) { lidx[d] = r % tl.ts[d]; r /= tl.ts[d]; }
            bool in = true;
            int lo = 0;
            int64_t gflat = 0;
            for (int d = 0; d < D; ++d) {
                if (lidx[d] >= e[d]) in = false;
                lo += lidx[d] * L.ls[d];
                gflat = gflat * geo.g[d] + o[d] + lidx[d];
            }
            const float* pl = sacc + (size_t)c * 2 * L.plane;
            float2 v = make_float2(pl[lo], pl[L.plane + lo]);
            if (slot < 0) {
                if (in) grid[(size_t)(c0 + c) * geo.G + gflat] = v;
            } else {
                partial[((size_t)slot * geo.C + c0 + c) * L.P + (i % L.P)] = v;
            }
        }
        __syncthreads();
    }
}

// Sum the partial tiles of split tiles into the grid.
template <int D>
__global__ void k_spread_reduce(const int* __restrict__ slot_off, const int* __restrict__ nslots,
                                const float2* __restrict__ partial, Geom geo, Tiles tl, int P,
                                float2* __restrict__ grid) {
    const int tile = blockIdx.x;
    const int ns = nslots[tile];
    if (ns == 0) return;
    const int s0 = slot_off[tile];
    int o[MAXD], e[MAXD];
    {
        int r = tile;
        for (int d = D - 1; d >= 0; --d) {
            int tc = r % tl.nt[d];
            r /= tl.nt[d];
            o[d] = tc * tl.ts[d];
            e[d] = min(tl.ts[d], geo.g[d] - o[d]);
        }
    }
    for (int i = threadIdx.x; i < geo.C * P; i += blockDim.x) {
        const int c = i / P;
        int r = i % P;
        int lidx[MAXD];
        for (int d = D - 1; d >= 0; --d) { lidx[d] = r % tl.ts[d]; r /= tl.ts[d]; }
        bool in = true;
        int64_t gflat = 0;
        for (int d = 0; d < D; ++d) {
            if (lidx[d] >= e[d]) in = false;
            gflat = gflat * geo.g[d] + o[d] + lidx[d];
        }
        if (!in) continue;
        float2 acc = make_float2(0.f, 0.f);
        for (int k = 0; k < ns; ++k) {
            float2 v = partial[((size_t)(s0 + k) * geo.C + c) * P + (i % P)];
            acc.x += v.x;
            acc.y += v.y;
        }
        grid[(size_t)c * geo.G + gflat] = acc;
    }
}

// ---------------------------------------------------------------- adjoint: post
template <int D, typename MT>
__device__ __forceinline__ float2 adj_pixel(const float2* __restrict__ grid, const MT* __restrict__ maps,
                                            const float* __restrict__ apod, const Geom& geo, int64_t j) {
    int jj[D];
    int64_t r = j;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) { jj[d] = (int)(r % geo.n[d]); r /= geo.n[d]; }
    int64_t gi = 0;
    float a = geo.rsqrtN;
    int ao = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        int nd = jj[d] - geo.n[d] / 2;
        int id = nd < 0 ? nd + geo.g[d] : nd;
        gi = gi * geo.g[d] + id;
        a *= apod[ao + jj[d]];
        ao += geo.n[d];
    }
    float2 acc = make_float2(0.f, 0.f);
    for (int c = 0; c < geo.C; ++c) {
        float2 gv = grid[(size_t)c * geo.G + gi];
        if (maps) {
            float2 s = ldc<MT>(maps, (size_t)c * geo.N + j);
            float2 v = cmulc(s, gv);
            acc.x += v.x;
            acc.y += v.y;
        } else {
            acc.x += gv.x;
            acc.y += gv.y;
        }
    }
    return make_float2(acc.x * a, acc.y * a);
}

template <int D, typename MT>
__global__ void k_adj_image(const float2* __restrict__ grid, const MT* __restrict__ maps, const float* __restrict__ apod,
                            Geom geo, float2* __restrict__ x) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= geo.N) return;
    x[j] = adj_pixel<D, MT>(grid, maps, apod, geo, j);
}

// Primal step (Sec. 4.1): z = x - tau A^H u; l2 prox z/(1 + tau lambda) and extrapolation
// fused (REG == 0); for the wavelet prox (REG == 1) z is written for the DWT.
template <int D, typename MT, int REG>
__global__ void k_adj_primal(const float2* __restrict__ grid, const MT* __restrict__ maps, const float* __restrict__ apod,
                             Geom geo, float2* __restrict__ x, float2* __restrict__ xbar, float2* __restrict__ z,
                             const float* __restrict__ sched, const int* __restrict__ iter, float lambda) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= geo.N) return;
    const int k = *iter;
    const float tau = sched[3 * k + 1], theta = sched[3 * k + 2];
    float2 ah = adj_pixel<D, MT>(grid, maps, apod, geo, j);
    float2 xo = x[j];
    float2 zz = make_float2(xo.x - tau * ah.x, xo.y - tau * ah.y);
    if (REG == 0) {
        float sc = 1.f / (1.f + tau * lambda);
        float2 xn = make_float2(zz.x * sc, zz.y * sc);
        xbar[j] = make_float2(xn.x + theta * (xn.x - xo.x), xn.y + theta * (xn.y - xo.y));
        x[j] = xn;
    } else {
        z[j] = zz;
    }
}

__global__ void k_fill(float2* __restrict__ x, int64_t n, float2 v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

// ---------------------------------------------------------------- host wrappers
#define KP_DISPATCH_T(tv, T, ...)                                                 \
    switch (tv) {                                                                 \
        case KP_C64: { using T = float2; __VA_ARGS__; } break;                    \
        case KP_C32_BF16: { using T = __nv_bfloat162; __VA_ARGS__; } break;       \
        case KP_C32_FP16: { using T = __half2; __VA_ARGS__; } break;              \
        default: set_error("bad complex storage type"); return KP_EINVAL;         \
    }

#define KP_DISPATCH_D(dv, DD, ...)                                                \
    if ((dv) == 2) { constexpr int DD = 2; __VA_ARGS__; }                         \
    else { constexpr int DD = 3; __VA_ARGS__; }

kp_status fill_image(float2* x, int64_t n, float2 v, cudaStream_t st) {
    k_fill<<<nblk(n, 256), 256, 0, st>>>(x, n, v);
    KP_LAUNCH_CHECK();
    return KP_OK;
}

static kp_status fwd_grid(kp_plan p, const float2* x, cudaStream_t st) {
    const Geom& g = p->geo;
    const kp_cdtype mt = p->unit_maps ? KP_C64 : p->maps_t;
    mark(p, PH_FWD_PRE, st);
    p->launches += 1;
    KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(mt, MT,
        k_fwd_pre<DD, MT><<<nblk(g.G, 256), 256, 0, st>>>(x, p->unit_maps ? nullptr : (const MT*)p->d_maps,
                                                         p->d_apod, g, p->d_grid)));
    KP_LAUNCH_CHECK();
    mark(p, PH_FFT_FWD, st);
    KP_TRY_CUFFT(cufftSetStream(p->fft, st));
    KP_TRY_CUFFT(cufftExecC2C(p->fft, (cufftComplex*)p->d_grid, (cufftComplex*)p->d_grid, CUFFT_FORWARD));
    return KP_OK;
}

kp_status forward_to(kp_plan p, const float2* x, void* out, kp_cdtype out_t, const int* perm, cudaStream_t st) {
    KP_TRY(fwd_grid(p, x, st));
    const Geom& g = p->geo;
    mark(p, PH_INTERP, st);
    p->launches += 1;
    KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(out_t, OT,
        k_interp_out<DD, OT><<<nblk(g.M, 128), 128, 0, st>>>(p->d_t, p->d_grid, g, perm, (OT*)out)));
    KP_LAUNCH_CHECK();
    return KP_OK;
}

kp_status forward_scaled(kp_plan p, const float2* x, float2* out_sorted, const float* ps, cudaStream_t st) {
    KP_TRY(fwd_grid(p, x, st));
    const Geom& g = p->geo;
    mark(p, PH_INTERP, st);
    p->launches += 1;
    KP_DISPATCH_D(g.D, DD, k_interp_scaled<DD><<<nblk(g.M, 128), 128, 0, st>>>(p->d_t, p->d_grid, g, ps, out_sorted));
    KP_LAUNCH_CHECK();
    return KP_OK;
}

kp_status forward_dual(kp_plan p, const float2* xbar, cudaStream_t st) {
    KP_TRY(fwd_grid(p, xbar, st));
    const Geom& g = p->geo;
    mark(p, PH_INTERP, st);
    p->launches += 1;
    KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(p->ys_t, YT,
        k_interp_dual<DD, YT><<<nblk(g.M, 128), 128, 0, st>>>(p->d_t, p->d_grid, g, (const YT*)p->d_ys, p->d_ps,
                                                             p->d_u, p->d_sched, p->d_iter)));
    KP_LAUNCH_CHECK();
    return KP_OK;
}

kp_status adjoint_to_grid(kp_plan p, const void* u, kp_cdtype u_t, const int* perm, cudaStream_t st) {
    const Geom& g = p->geo;
    const SpreadLayout L = spread_layout(p->tiles, g.D);
    const int cc = g.C < SP_CH ? g.C : SP_CH;
    const size_t smem = (size_t)cc * 2 * L.plane * sizeof(float);
    static bool attr_set[2][3] = {{false}};
    mark(p, PH_SPREAD, st);
    p->launches += 1;
    KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(u_t, UT,
        if (!attr_set[DD - 2][u_t]) {
            KP_TRY_CUDA(cudaFuncSetAttribute(k_spread<DD, UT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
            attr_set[DD - 2][u_t] = true;
        }
        k_spread<DD, UT><<<(unsigned)p->n_items, SP_THREADS, smem, st>>>(p->d_t, (const UT*)u, perm, p->d_ext,
                                                                        p->d_items, g, p->tiles, L, p->d_grid,
                                                                        p->d_partial)));
    KP_LAUNCH_CHECK();
    if (p->n_slots > 0) {
        mark(p, PH_SPREAD_RED, st);
        p->launches += 1;
        KP_DISPATCH_D(g.D, DD, k_spread_reduce<DD><<<(unsigned)p->tiles.ntiles, 256, 0, st>>>(
            p->d_slot_off, p->d_nslots, p->d_partial, g, p->tiles, L.P, p->d_grid));
        KP_LAUNCH_CHECK();
    }
    mark(p, PH_FFT_INV, st);
    KP_TRY_CUFFT(cufftSetStream(p->fft, st));
    KP_TRY_CUFFT(cufftExecC2C(p->fft, (cufftComplex*)p->d_grid, (cufftComplex*)p->d_grid, CUFFT_INVERSE));
    return KP_OK;
}

kp_status grid_to_image(kp_plan p, float2* x, cudaStream_t st) {
    const Geom& g = p->geo;
    const kp_cdtype mt = p->unit_maps ? KP_C64 : p->maps_t;
    mark(p, PH_ADJ, st);
    p->launches += 1;
    KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(mt, MT,
        k_adj_image<DD, MT><<<nblk(g.N, 256), 256, 0, st>>>(p->d_grid, p->unit_maps ? nullptr : (const MT*)p->d_maps,
                                                           p->d_apod, g, x)));
    KP_LAUNCH_CHECK();
    return KP_OK;
}

kp_status adjoint_primal(kp_plan p, int reg, float lambda, cudaStream_t st) {
    const Geom& g = p->geo;
    const kp_cdtype mt = p->unit_maps ? KP_C64 : p->maps_t;
    mark(p, PH_ADJ, st);
    p->launches += 1;
    if (reg == KP_REG_L2) {
        KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(mt, MT,
            k_adj_primal<DD, MT, 0><<<nblk(g.N, 256), 256, 0, st>>>(p->d_grid, (const MT*)p->d_maps, p->d_apod, g, p->d_x,
                                                                   p->d_xbar, p->d_z, p->d_sched, p->d_iter, lambda)));
    } else {
        KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(mt, MT,
            k_adj_primal<DD, MT, 1><<<nblk(g.N, 256), 256, 0, st>>>(p->d_grid, (const MT*)p->d_maps, p->d_apod, g, p->d_x,
                                                                   p->d_xbar, p->d_z, p->d_sched, p->d_iter, lambda)));
    }
    KP_LAUNCH_CHECK();
    return KP_OK;
}

}  // namespace kp

using namespace kp;

extern "C" {

kp_status kp_sense_forward(kp_plan plan, const void* x_dev, void* y_dev, kp_cdtype y_t, void* stream) {
    if (!plan || !x_dev || !y_dev) { set_error("null argument"); return KP_EINVAL; }
    if (!plan->traj_set || (!plan->maps_set && !plan->unit_maps)) { set_error("trajectory and maps must be set"); return KP_EINVAL; }
    if (y_t != KP_C64 && y_t != KP_C32_BF16 && y_t != KP_C32_FP16) { set_error("bad y type"); return KP_EINVAL; }
    return forward_to(plan, (const float2*)x_dev, y_dev, y_t, plan->d_perm, (cudaStream_t)stream);
}

kp_status kp_sense_adjoint(kp_plan plan, const void* y_dev, kp_cdtype y_t, void* x_dev, void* stream) {
    if (!plan || !x_dev || !y_dev) { set_error("null argument"); return KP_EINVAL; }
    if (!plan->traj_set || (!plan->maps_set && !plan->unit_maps)) { set_error("trajectory and maps must be set"); return KP_EINVAL; }
    if (y_t != KP_C64 && y_t != KP_C32_BF16 && y_t != KP_C32_FP16) { set_error("bad y type"); return KP_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    KP_TRY(adjoint_to_grid(plan, y_dev, y_t, plan->d_perm, st));
    return grid_to_image(plan, (float2*)x_dev, st);
}

}  // extern "C"
