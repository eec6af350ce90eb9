// Multi-coil SENSE NUFFT pair A = F_nu S and A^H on sm_103a (Sec. 2 Eq. model_i;
// Sec. 6: Kaiser-Bessel gridding following Beatty et al., oversampling g/n, width 4).
//
// Forward:  fwd_pre (coil multiply, 1/Phi apodisation, centred zero padding; writes the
//           whole grid) -> cuFFT C2C forward, batch C -> interp (W^D taps per sample,
//           one thread per sorted sample, all coils, N^{-1/2}).
// Adjoint:  spread into a second grid (one CTA per (tile, chunk) work item; each sample is
//           taken by a group of lanes, one lane per tap, looping over coils, so shared-memory
//           atomics of one sample never collide; single-chunk tiles store straight to the
//           grid, chunks of split tiles add their tile with global atomics into a region
//           cleared just before) -> cuFFT C2C inverse -> adj_post (crop, 1/Phi, conj(s_c)
//           coil combine, N^{-1/2}).
// The Kaiser-Bessel weights and first taps of every sample are tabulated once per
// trajectory (sorted order, structure of arrays), so no Bessel function is evaluated
// inside the iteration.
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
__device__ __forceinline__ void make_taps(const int* __restrict__ k0t, const float* __restrict__ wt, int64_t s,
                                          const Geom& geo, Taps<D>& tp) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int k0w = k0t[(int64_t)d * geo.M + s];
        int stride = 1;
        for (int e = d + 1; e < D; ++e) stride *= geo.g[e];
#pragma unroll
        for (int j = 0; j < KW; ++j) {
            int ix = k0w + j;
            if (ix >= geo.g[d]) ix -= geo.g[d];
            tp.w[d][j] = wt[(int64_t)(d * KW + j) * geo.M + s];
            tp.idx[d][j] = ix;
            tp.off[d][j] = ix * stride;
        }
    }
}

// Tap tables of the sorted samples: wrapped first tap k0 = ceil(t) - W/2 (mod g) and the
// Kaiser-Bessel weights phi(t - k) of the W taps per axis.
template <int D>
__global__ void k_tap_tables(const float* __restrict__ t, Geom geo, int* __restrict__ k0t, float* __restrict__ wt) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= geo.M) return;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const float td = t[(int64_t)d * geo.M + s];
        const int k0 = (int)ceilf(td) - KW / 2;
        k0t[(int64_t)d * geo.M + s] = wrapg(k0, geo.g[d]);
#pragma unroll
        for (int j = 0; j < KW; ++j) wt[(int64_t)(d * KW + j) * geo.M + s] = kbw(td - (float)(k0 + j), geo.beta[d]);
    }
}

kp_status build_tap_tables(kp_plan p, cudaStream_t st) {
    const Geom& g = p->geo;
    if (g.D == 2) k_tap_tables<2><<<nblk(g.M, 256), 256, 0, st>>>(p->d_t, g, p->d_k0, p->d_wt);
    else k_tap_tables<3><<<nblk(g.M, 256), 256, 0, st>>>(p->d_t, g, p->d_k0, p->d_wt);
    KP_LAUNCH_CHECK();
    p->launches += 1;
    return KP_OK;
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

// ---------------------------------------------------------------- forward: interpolation
// One CTA per (tile chunk, coil group): the grid region the tile's samples read
// ((ts + W - 1)^D points per coil, periodic) is staged in shared memory with coalesced loads,
// then each thread interpolates one sample for the group's coils from shared memory.
constexpr int IP_CH = 4;           // coils per CTA (blockIdx.y selects the group)
constexpr int IP_THREADS = 256;

struct InterpIO {
    void* out;           // mode 0: [C][M] storage type T, index perm[s] (or s)
    const int* perm;
    float2* outs;        // mode 1: [C][M] sorted, scaled by p
    const float* ps;     // modes 1, 2: sorted preconditioner
    const void* ys;      // mode 2: sorted measurements, storage type T
    float2* u;           // mode 2: dual variable, sorted
    const float* sched;
    const int* iter;
};

template <int D, int MODE, typename T>
__global__ void __launch_bounds__(IP_THREADS)
k_interp_tile(const int4* __restrict__ items, const int* __restrict__ k0t, const float* __restrict__ wt,
              const float2* __restrict__ grid, Geom geo, Tiles tl, InterpIO io) {
    extern __shared__ float2 sg[];    // [IP_CH][R^D]
    const int4 it = items[blockIdx.x];
    const int tile = it.x, beg = it.y, end = it.z;
    const int c0 = blockIdx.y * IP_CH;
    const int cc = min(IP_CH, geo.C - c0);
    int o[MAXD], R[MAXD], rs[MAXD];
    {
        int r = tile;
        for (int d = D - 1; d >= 0; --d) {
            const int tc = r % tl.nt[d];
            r /= tl.nt[d];
            o[d] = tc * tl.ts[d];
            R[d] = tl.ts[d] + KW - 1;
        }
        int st = 1;
        for (int d = D - 1; d >= 0; --d) { rs[d] = st; st *= R[d]; }
    }
    int Rtot = 1;
    for (int d = 0; d < D; ++d) Rtot *= R[d];
    for (int idx = threadIdx.x; idx < cc * Rtot; idx += blockDim.x) {
        const int c = idx / Rtot;
        int r = idx - c * Rtot;
        int64_t flat = 0;
        int lrev[MAXD];
        for (int d = D - 1; d >= 0; --d) { lrev[d] = r % R[d]; r /= R[d]; }
        for (int d = 0; d < D; ++d) {
            int pp = o[d] + lrev[d];
            if (pp >= geo.g[d]) pp -= geo.g[d];
            flat = flat * geo.g[d] + tunshift(pp, tl.sh[d], geo.g[d]);
        }
        sg[c * Rtot + (idx - c * Rtot)] = __ldg(grid + (size_t)(c0 + c) * geo.G + flat);
    }
    __syncthreads();
    float sigma = 0.f;
    if (MODE == 2) sigma = io.sched[3 * (*io.iter)];
    for (int s = beg + threadIdx.x; s < end; s += blockDim.x) {
        float w[D][KW];
        int lb = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int p0 = tshift(k0t[(int64_t)d * geo.M + s], tl.sh[d], geo.g[d]);
            lb += (p0 - o[d]) * rs[d];
#pragma unroll
            for (int j = 0; j < KW; ++j) w[d][j] = wt[(int64_t)(d * KW + j) * geo.M + s];
        }
        for (int c = 0; c < cc; ++c) {
            const float2* base = sg + c * Rtot + lb;
            float2 acc = make_float2(0.f, 0.f);
            if (D == 2) {
#pragma unroll
                for (int a = 0; a < KW; ++a)
#pragma unroll
                    for (int b = 0; b < KW; ++b) {
                        const float ww = w[0][a] * w[D - 1][b];
                        const float2 v = base[a * rs[0] + b];
                        acc.x = fmaf(ww, v.x, acc.x);
                        acc.y = fmaf(ww, v.y, acc.y);
                    }
            } else {
#pragma unroll
                for (int a = 0; a < KW; ++a)
#pragma unroll
                    for (int b = 0; b < KW; ++b) {
                        const float wab = w[0][a] * w[1 % D][b];
#pragma unroll
                        for (int e = 0; e < KW; ++e) {
                            const float ww = wab * w[D - 1][e];
                            const float2 v = base[a * rs[0] + b * rs[1 % D] + e];
                            acc.x = fmaf(ww, v.x, acc.x);
                            acc.y = fmaf(ww, v.y, acc.y);
                        }
                    }
            }
            acc.x *= geo.rsqrtN;
            acc.y *= geo.rsqrtN;
            const size_t os = (size_t)(c0 + c) * geo.M + s;
            if (MODE == 0) {
                const int64_t oi = io.perm ? io.perm[s] : s;
                stc<T>((T*)io.out, (size_t)(c0 + c) * geo.M + oi, acc);
            } else if (MODE == 1) {
                const float sc = io.ps ? io.ps[os] : 1.f;
                io.outs[os] = make_float2(acc.x * sc, acc.y * sc);
            } else {
                // PDHG dual step (Sec. 4.1): u <- (u + sigma p (A xbar - y)) / (1 + sigma p)
                const float2 y = ldc<T>((const T*)io.ys, os);
                const float sp = sigma * io.ps[os];
                const float inv = 1.f / (1.f + sp);
                const float2 uo = io.u[os];
                io.u[os] = make_float2((uo.x + sp * (acc.x - y.x)) * inv, (uo.y + sp * (acc.y - y.y)) * inv);
            }
        }
    }
}

// ---------------------------------------------------------------- adjoint: spread
// One CTA per (spreading work item, coil group).  The item's samples (their coil values,
// first taps and weights) are staged in shared memory by all threads at once; then each
// warp takes one sample at a time, its lanes covering distinct (tap, coil) pairs, and adds
// into its own private copy of the tile, so no atomics are needed.  The private copies are
// summed and the tile is stored (or, for a tile split over several items, added with global
// atomics into a region cleared beforehand).  Tile coordinates are shifted (Tiles::sh).
constexpr int SP_CH = 4;           // coils per CTA
constexpr int SP_THREADS = 128;    // 4 warps, 4 private tile copies
constexpr int SP_CHUNK = 256;      // samples per work item (== plan chunk)

struct SpreadLayout {
    int ls[MAXD];      // shared-memory strides of the local tile index
    int plane;         // floats per (warp, coil, re/im) plane
    int P;             // tile points
};

static SpreadLayout spread_layout(const Tiles& tl, int D) {
    SpreadLayout L{};
    int st = 1;
    for (int d = D - 1; d >= 0; --d) { L.ls[d] = st; st *= tl.ts[d]; }
    L.P = st;
    L.plane = st;
    return L;
}

template <int D, typename UT>
__global__ void __launch_bounds__(SP_THREADS)
k_spread(const int* __restrict__ k0t, const float* __restrict__ wt, const UT* __restrict__ u,
         const int* __restrict__ perm, const int* __restrict__ ext, const int4* __restrict__ items, Geom geo,
         Tiles tl, SpreadLayout L, float2* __restrict__ grid) {
    extern __shared__ float smem[];
    constexpr int NW = SP_THREADS / 32;
    float* acc = smem;                                              // [NW][SP_CH][2][P]
    float2* su = (float2*)(acc + NW * SP_CH * 2 * L.plane);         // [SP_CHUNK][SP_CH]
    float* sw = (float*)(su + SP_CHUNK * SP_CH);                    // [SP_CHUNK][D*KW]
    int* sl = (int*)(sw + SP_CHUNK * D * KW);                       // [SP_CHUNK][D] local first tap (may be < 0)
    const int4 it = items[blockIdx.x];
    const int tile = it.x, beg = it.y, end = it.z;
    const bool split = it.w >= 0;
    const int c0 = blockIdx.y * SP_CH;
    const int cc = min(SP_CH, geo.C - c0);
    int o[MAXD], e[MAXD];
    {
        int r = tile;
        for (int d = D - 1; d >= 0; --d) {
            const int tc = r % tl.nt[d];
            r /= tl.nt[d];
            o[d] = tc * tl.ts[d];
            e[d] = min(tl.ts[d], geo.g[d] - o[d]);
        }
    }
    const int n = end - beg;
    for (int i = threadIdx.x; i < NW * SP_CH * 2 * L.plane; i += blockDim.x) acc[i] = 0.f;
    // stage the item's samples
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int s = ext[beg + i];
        const int64_t un = perm ? perm[s] : s;
#pragma unroll
        for (int c = 0; c < SP_CH; ++c)
            su[i * SP_CH + c] = c < cc ? ldc<UT>(u, (size_t)(c0 + c) * geo.M + un) : make_float2(0.f, 0.f);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            int p0 = tshift(k0t[(int64_t)d * geo.M + s], tl.sh[d], geo.g[d]) - o[d];
            // the footprint may start in the previous tile (or wrap around the axis)
            if (p0 > e[d]) p0 -= geo.g[d];
            sl[i * D + d] = p0;
#pragma unroll
            for (int j = 0; j < KW; ++j) sw[i * D * KW + d * KW + j] = wt[(int64_t)(d * KW + j) * geo.M + s];
        }
    }
    __syncthreads();
    constexpr int TAPS = D == 2 ? KW * KW : KW * KW * KW;
    constexpr int LPT = TAPS < 32 ? 32 / TAPS : 1;     // lanes per tap (2D: 2, coils split between them)
    constexpr int TPL = TAPS > 32 ? TAPS / 32 : 1;     // taps per lane (3D: 2)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* my = acc + warp * SP_CH * 2 * L.plane;
    for (int i = warp; i < n; i += NW) {
#pragma unroll
        for (int tq = 0; tq < TPL; ++tq) {
            int q = (TAPS < 32 ? lane % TAPS : lane) + 32 * tq;
            float w = 1.f;
            int lo = 0;
            bool ok = true;
#pragma unroll
            for (int d = D - 1; d >= 0; --d) {
                const int j = q % KW;
                q /= KW;
                int pp = o[d] + sl[i * D + d] + j;      // shifted coordinate of the tap
                if (pp < 0) pp += geo.g[d];
                else if (pp >= geo.g[d]) pp -= geo.g[d];
                const int l = pp - o[d];
                if (l < 0 || l >= e[d]) ok = false;
                w *= sw[i * D * KW + d * KW + j];
                lo += l * L.ls[d];
            }
            if (!ok) continue;
            for (int c = (TAPS < 32 ? lane / TAPS : 0); c < cc; c += LPT) {
                const float2 uv = su[i * SP_CH + c];
                float* pl = my + c * 2 * L.plane;
                pl[lo] += w * uv.x;
                pl[L.plane + lo] += w * uv.y;
            }
        }
        __syncwarp();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cc * L.P; i += blockDim.x) {
        const int c = i / L.P;
        const int r0 = i - c * L.P;
        int r = r0;
        int lidx[MAXD];
        for (int d = D - 1; d >= 0; --d) { lidx[d] = r % tl.ts[d]; r /= tl.ts[d]; }
        bool in = true;
        int64_t gflat = 0;
        for (int d = 0; d < D; ++d) {
            if (lidx[d] >= e[d]) in = false;
            gflat = gflat * geo.g[d] + tunshift(o[d] + lidx[d], tl.sh[d], geo.g[d]);
        }
        if (!in) continue;
        float2 v = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const float* pl = acc + (w * SP_CH + c) * 2 * L.plane;
            v.x += pl[r0];
            v.y += pl[L.plane + r0];
        }
        float2* dst = grid + (size_t)(c0 + c) * geo.G + gflat;
        if (split) {
            atomicAdd(&dst->x, v.x);
            atomicAdd(&dst->y, v.y);
        } else {
            *dst = v;
        }
    }
}

// Clear the grid region of every split tile (all coils) before the spreading kernel adds
// the tile's chunks into it.
template <int D>
__global__ void k_zero_split(const int* __restrict__ split_tiles, Geom geo, Tiles tl, int P, float2* __restrict__ grid) {
    const int tile = split_tiles[blockIdx.x];
    int o[MAXD], e[MAXD];
    {
        int r = tile;
        for (int d = D - 1; d >= 0; --d) {
            const int tc = r % tl.nt[d];
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
            gflat = gflat * geo.g[d] + tunshift(o[d] + lidx[d], tl.sh[d], geo.g[d]);
        }
        if (in) grid[(size_t)c * geo.G + gflat] = make_float2(0.f, 0.f);
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

template <int MODE>
static kp_status launch_interp(kp_plan p, kp_cdtype t, const InterpIO& io, cudaStream_t st) {
    const Geom& g = p->geo;
    size_t rt = 1;
    for (int d = 0; d < g.D; ++d) rt *= p->tiles.ts[d] + KW - 1;
    const size_t smem = (size_t)IP_CH * rt * sizeof(float2);
    const dim3 grid((unsigned)p->n_iitems, (g.C + IP_CH - 1) / IP_CH);
    static bool attr[2][3][3] = {};
    mark(p, PH_INTERP, st);
    p->launches += 1;
    if (p->n_iitems == 0) return KP_OK;
    KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(t, T,
        if (!attr[DD - 2][MODE][t]) {
            KP_TRY_CUDA(cudaFuncSetAttribute(k_interp_tile<DD, MODE, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
            attr[DD - 2][MODE][t] = true;
        }
        k_interp_tile<DD, MODE, T><<<grid, IP_THREADS, smem, st>>>(p->d_iitems, p->d_k0, p->d_wt, p->d_grid, g, p->tiles, io)));
    KP_LAUNCH_CHECK();
    return KP_OK;
}

kp_status forward_to(kp_plan p, const float2* x, void* out, kp_cdtype out_t, const int* perm, cudaStream_t st) {
    KP_TRY(fwd_grid(p, x, st));
    InterpIO io{};
    io.out = out;
    io.perm = perm;
    return launch_interp<0>(p, out_t, io, st);
}

kp_status forward_scaled(kp_plan p, const float2* x, float2* out_sorted, const float* ps, cudaStream_t st) {
    KP_TRY(fwd_grid(p, x, st));
    InterpIO io{};
    io.outs = out_sorted;
    io.ps = ps;
    return launch_interp<1>(p, KP_C64, io, st);
}

kp_status forward_dual(kp_plan p, const float2* xbar, cudaStream_t st) {
    KP_TRY(fwd_grid(p, xbar, st));
    InterpIO io{};
    io.ys = p->d_ys;
    io.ps = p->d_ps;
    io.u = p->d_u;
    io.sched = p->d_sched;
    io.iter = p->d_iter;
    return launch_interp<2>(p, p->ys_t, io, st);
}

kp_status adjoint_to_grid(kp_plan p, const void* u, kp_cdtype u_t, const int* perm, cudaStream_t st) {
    const Geom& g = p->geo;
    const SpreadLayout L = spread_layout(p->tiles, g.D);
    const size_t smem = (size_t)(SP_THREADS / 32) * SP_CH * 2 * L.plane * sizeof(float) +
                        (size_t)SP_CHUNK * (SP_CH * sizeof(float2) + g.D * KW * sizeof(float) + g.D * sizeof(int));
    static bool attr_set[2][3] = {{false}};
    mark(p, PH_SPREAD, st);
    if (p->n_split > 0) {
        KP_DISPATCH_D(g.D, DD, k_zero_split<DD><<<(unsigned)p->n_split, 256, 0, st>>>(p->d_split, g, p->tiles, L.P,
                                                                                      p->d_grid2));
        KP_LAUNCH_CHECK();
        p->launches += 1;
    }
    p->launches += 1;
    KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(u_t, UT,
        if (!attr_set[DD - 2][u_t]) {
            KP_TRY_CUDA(cudaFuncSetAttribute(k_spread<DD, UT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
            attr_set[DD - 2][u_t] = true;
        }
        k_spread<DD, UT><<<dim3((unsigned)p->n_items, (g.C + SP_CH - 1) / SP_CH), SP_THREADS, smem, st>>>(p->d_k0, p->d_wt, (const UT*)u, perm, p->d_ext,
                                                                        p->d_items, g, p->tiles, L, p->d_grid2)));
    KP_LAUNCH_CHECK();
    mark(p, PH_FFT_INV, st);
    KP_TRY_CUFFT(cufftSetStream(p->fft, st));
    KP_TRY_CUFFT(cufftExecC2C(p->fft, (cufftComplex*)p->d_grid2, (cufftComplex*)p->d_grid2, CUFFT_INVERSE));
    return KP_OK;
}

kp_status grid_to_image(kp_plan p, float2* x, cudaStream_t st) {
    const Geom& g = p->geo;
    const kp_cdtype mt = p->unit_maps ? KP_C64 : p->maps_t;
    mark(p, PH_ADJ, st);
    p->launches += 1;
    KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(mt, MT,
        k_adj_image<DD, MT><<<nblk(g.N, 256), 256, 0, st>>>(p->d_grid2, p->unit_maps ? nullptr : (const MT*)p->d_maps,
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
            k_adj_primal<DD, MT, 0><<<nblk(g.N, 256), 256, 0, st>>>(p->d_grid2, (const MT*)p->d_maps, p->d_apod, g, p->d_x,
                                                                   p->d_xbar, p->d_z, p->d_sched, p->d_iter, lambda)));
    } else {
        KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(mt, MT,
            k_adj_primal<DD, MT, 1><<<nblk(g.N, 256), 256, 0, st>>>(p->d_grid2, (const MT*)p->d_maps, p->d_apod, g, p->d_x,
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
