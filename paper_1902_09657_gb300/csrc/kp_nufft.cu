// Multi-coil SENSE NUFFT pair A = F_nu S and A^H on sm_103a (Sec. 2 Eq. model_i;
// Sec. 6: Kaiser-Bessel gridding following Beatty et al., oversampling g/n, width 4).
//
// Forward:  pre-step (coil multiply, 1/Phi apodisation, centred zero padding) -> forward FFT
//           of every coil's grid (2D: cuFFT; 3D: the own passes of kp_fft.cu, whose first pass
//           forms the pre-step itself) -> interpolation (one CTA per (tile item, 4 coils), the
//           tile's grid region staged in shared memory, one thread per sorted sample, W^D taps,
//           N^{-1/2}).
// Adjoint:  spreading into a second grid (variants chosen per plan by the autotuner: private
//           tile copies per warp, or in 3D the two-phase padded tiles + gather; no zero-fill of
//           the grid, split tiles cleared before they are accumulated) -> inverse FFT (cuFFT or
//           the own passes, which leave only the crop valid) -> crop, 1/Phi, conj(s_c) coil
//           combine, N^{-1/2} (fused into the primal step inside a PDHG iteration).
// The Kaiser-Bessel weights and first taps of every sample are tabulated once per
// trajectory (sorted order, structure of arrays), so no Bessel function is evaluated
// inside the iteration.
// The grid coordinates t = f g/n are formed in float64 at binning (grid_tap); the first tap is
// k0 = ceil(t) - W/2, which equals ceil(t - W/2) exactly, so |t - k| <= W/2 for every tap, and
// the weights come from the float32 offset t - ceil(t).
#include "kp_internal.cuh"

#include <cstdlib>
#include <vector>

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

// Kaiser-Bessel weights of the sorted samples: phi(t - k) for the W taps per axis, from the
// offset u0 = t - ceil(t) written by the binning (t - (k0 + j) = u0 + W/2 - j).
template <int D>
__global__ void k_tap_tables(const float* __restrict__ u0t, Geom geo, float* __restrict__ wt) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= geo.M) return;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const float u0 = u0t[(int64_t)d * geo.M + s];
#pragma unroll
        for (int j = 0; j < KW; ++j) wt[(int64_t)(d * KW + j) * geo.M + s] = kbw(u0 + (float)(KW / 2 - j), geo.beta[d]);
    }
}

kp_status build_tap_tables(kp_plan p, cudaStream_t st) {
    const Geom& g = p->geo;
    if (g.D == 2) k_tap_tables<2><<<nblk(g.M, 256), 256, 0, st>>>(p->d_t, g, p->d_wt);
    else k_tap_tables<3><<<nblk(g.M, 256), 256, 0, st>>>(p->d_t, g, p->d_wt);
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
__device__ __forceinline__ void fwd_pre_body(const float2* __restrict__ x, const MT* __restrict__ maps,
                                             const float* __restrict__ apod, const Geom& geo,
                                             float2* __restrict__ grid, int64_t gi) {
    if (gi >= geo.G) return;
    int ii[D];
    if (geo.G < ((int64_t)1 << 31)) {        // 32-bit index arithmetic (64-bit division is slow)
        unsigned r = (unsigned)gi;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { ii[d] = (int)(r % (unsigned)geo.g[d]); r /= (unsigned)geo.g[d]; }
    } else {
        int64_t r = gi;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { ii[d] = (int)(r % geo.g[d]); r /= geo.g[d]; }
    }
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
    if (!KP_INB(11, j, geo.N)) return;
    float2 xv = x[j];
    xv.x *= a;
    xv.y *= a;
    for (int c = 0; c < geo.C; ++c) {
        float2 s = maps ? ldc<MT>(maps, (size_t)c * geo.N + j) : make_float2(1.f, 0.f);
        grid[(size_t)c * geo.G + gi] = cmul(s, xv);
    }
}

template <int D, typename MT>
__global__ void k_fwd_pre(const float2* __restrict__ x, const MT* __restrict__ maps, const float* __restrict__ apod,
                          Geom geo, float2* __restrict__ grid) {
    fwd_pre_body<D, MT>(x, maps, apod, geo, grid, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------- forward: interpolation
// One CTA per (tile chunk, coil group): the grid region the tile's samples read
// ((ts + W - 1)^D points per coil, periodic) is staged in shared memory by bulk asynchronous
// copies (cp.async.bulk, one or two per grid row, completing on an mbarrier), then each
// thread interpolates one sample for the group's coils from shared memory.
constexpr int IP_CH = 4;           // coils per CTA (blockIdx.y selects the group)
constexpr int IP_THREADS = 256;     // four CTAs per SM (64 registers; 3D: 4 x 46.5 KB staged)

struct InterpIO {
    void* out;           // mode 0: [C][M] storage type T, index perm[s] (or s)
    const int* perm;
    float2* outs;        // mode 1: [C][M] sorted, scaled by p
    const float* ps;     // modes 1, 2: sorted preconditioner
    const void* ys;      // mode 2: sorted measurements, storage type T
    float2* u;           // mode 2: dual variable, sorted
    const float* sched;
    const int* iter;
    int* flag;           // set to 1 if the staging wait gave up (reported as KP_ETIMEOUT)
    const double* n2;    // mode 1: when set, the output is also divided by sqrt(*n2)
    long long wait;      // limit of the staging wait (SM clock cycles)
};

// Per-case arguments of the batched launches (one launch per phase over the cases of a batch;
// nx = the case's work items, so its blocks are nx x coil groups).
struct BInterp {
    const int4* items;
    const int* k0t;
    const float* wt;
    const float2* grid;
    Geom geo;
    Tiles tl;
    InterpIO io;
    int nx;
};
struct BSpread {
    const int* k0t;
    const float* wt;
    const void* u;
    const int* perm;
    const int* ext;
    const int4* items;
    Geom geo;
    Tiles tl;
    float2* grid;
    int nx;
};
struct BZero {
    const int* split;
    Geom geo;
    Tiles tl;
    int P;
    float2* grid;
};
struct BPrimal {             // reg 0: l2 prox + extrapolation; 1: z for the wavelet prox
    const float2* grid;
    const void* maps;
    const float* apod;
    Geom geo;
    float2* x;
    float2* xbar;
    float2* z;
    const float* sched;
    const int* iter;
    float lambda;
    int reg;
};
struct BPre {
    const float2* x;
    const void* maps;
    const float* apod;
    Geom geo;
    float2* grid;
};

// Staged region geometry: R points per axis for the largest tile edge (16 in 2D, 8 in 3D);
// rows along the last axis are copied RP points long (even, so every copy is a multiple of
// 16 bytes starting on a 16-byte boundary: the row start is rounded down to an even x).
template <int D> struct IpL {
    static constexpr int R = (D == 2 ? 16 : 8) + KW - 1;
    static constexpr int RP = (R + 2) & ~1;
    static constexpr int ROWS = D == 2 ? R : R * R;      // rows per coil
    static constexpr int PER_COIL = ROWS * RP;           // staged points per coil
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared.b64 st, [%0], %1; }"
                 :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile("{ .reg .pred p; mbarrier.test_wait.parity.shared.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Waits for phase `parity` of the barrier for at most `limit` SM clock cycles; false if it gave
// up.  A limit of 0 does not wait at all: a phase not yet complete gives up at once.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, long long limit) {
    if (mbar_test_wait(bar, parity)) return true;
    if (limit <= 0) return false;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Stages the periodic grid region an interpolation CTA reads ((ts + W - 1)^D points of coils
// c0 .. c0 + cc - 1, rows of RP points starting at an even x) into sg by bulk asynchronous row
// copies completing on `bar`; o receives the tile's origin and xo the parity of its first x.
// The caller waits on bar (bounded).
template <int D>
__device__ __forceinline__ void interp_stage(int tile, int c0, int cc, const float2* __restrict__ grid, const Geom& geo,
                                             const Tiles& tl, float2* sg, unsigned long long* bar, int* o, int& xo) {
    using LY = IpL<D>;
    constexpr int R = LY::R;
    {
        int r = tile;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            const int tc = r % tl.nt[d];
            r /= tl.nt[d];
            o[d] = tc * tl.ts[d];
        }
    }
    // grid row offsets of the staged region along the slower axes (periodic), computed once
    __shared__ int rowoff[MAXD][R];
    if (threadIdx.x < (D - 1) * R) {
        // axis d < D - 1 without indexing the parameter structs by a thread-dependent d
        const int d = threadIdx.x / R, l = threadIdx.x % R;
        const int gd = d == 0 ? geo.g[0] : geo.g[1];
        const int sd = d == 0 ? tl.sh[0] : tl.sh[1];
        const int od = d == 0 ? o[0] : o[1 % D];
        const int stride = D == 3 ? (d == 0 ? geo.g[1] * geo.g[2] : geo.g[2]) : (d == 0 ? geo.g[1] : 1);
        int pp = od + l;
        while (pp >= gd) pp -= gd;
        rowoff[d][l] = tunshift(pp, sd, gd) * stride;
    }
    // first staged x (unshifted), rounded down to even; xo = its parity
    const int gx = geo.g[D - 1];
    const int xs = tunshift(o[D - 1] < gx ? o[D - 1] : o[D - 1] - gx, tl.sh[D - 1], gx);
    xo = xs & 1;
    const int xlo = xs - xo;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, (unsigned)(cc * LY::PER_COIL * sizeof(float2)));
    for (int j = threadIdx.x; j < cc * LY::ROWS; j += blockDim.x) {
        const int c = j / LY::ROWS, row = j - c * LY::ROWS;
        const int off = D == 2 ? rowoff[0][row] : rowoff[0][row / R] + rowoff[1 % (D - 1)][row % R];
        const float2* src = grid + (size_t)(c0 + c) * geo.G + off;
        float2* dst = sg + (size_t)j * LY::RP;
        // the row is periodic: copy up to the grid edge, then continue from x = 0 (pieces
        // are even in length because the grid extent and the start are even)
        for (int pos = 0, x = xlo; pos < LY::RP; x = 0) {
            const int n = min(LY::RP - pos, gx - x);
            const int64_t o0 = (int64_t)(c0 + c) * geo.G + off + x;
            // (checked build: a piece out of range copies the grid's first points instead, so the
            // barrier still receives the bytes it expects)
            const bool ok = KP_INB(4, o0, (int64_t)geo.C * geo.G) && KP_INB(4, o0 + n - 1, (int64_t)geo.C * geo.G);
            bulk_g2s(dst + pos, ok ? src + x : grid, (unsigned)(n * sizeof(float2)), bar);
            pos += n;
        }
    }
}

template <int D, int MODE, typename T>
__device__ __forceinline__ void interp_tile_body(const int4* __restrict__ items, const int* __restrict__ k0t,
                                                 const float* __restrict__ wt, const float2* __restrict__ grid,
                                                 const Geom& geo, const Tiles& tl, const InterpIO& io, int bx, int by) {
    using LY = IpL<D>;
    extern __shared__ __align__(128) float2 sg[];    // [IP_CH][ROWS][RP]
    __shared__ unsigned long long bar;
    const int4 it = items[bx];
    const int tile = it.x, beg = it.y, end = it.z;
    const int c0 = by * IP_CH;
    const int cc = min(IP_CH, geo.C - c0);
    constexpr int R = LY::R;
    int o[MAXD], xo;
    interp_stage<D>(tile, c0, cc, grid, geo, tl, sg, &bar, o, xo);
    constexpr int rs0 = D == 2 ? LY::RP : R * LY::RP, rs1 = D == 2 ? 1 : LY::RP;
    constexpr int Rtot = LY::PER_COIL;
    // While the grid region is in flight: this thread's sample (items hold at most blockDim.x
    // samples), its tap tables and, for the dual step in 2D, its y, p and u.
    const int s = beg + (int)threadIdx.x;
    bool act = s < end && KP_INB(5, s, geo.M);
    float w[D][KW];
    int lb = xo;
    constexpr bool PRE = MODE == 2 && D == 2;     // 3D keeps registers for the 64 taps
    float2 yv[PRE ? IP_CH : 1], uv[PRE ? IP_CH : 1];
    float pv[PRE ? IP_CH : 1];
    float sigma = 0.f;
    if (act) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int p0 = tshift(k0t[(int64_t)d * geo.M + s], tl.sh[d], geo.g[d]);
            lb += (p0 - o[d]) * (d == 0 ? rs0 : (d == 1 ? rs1 : 1));
#pragma unroll
            for (int j = 0; j < KW; ++j) w[d][j] = wt[(int64_t)(d * KW + j) * geo.M + s];
        }
        // the footprint lies in the staged region (the sample's first tap is in this tile)
        act = KP_INB(4, lb, Rtot) && KP_INB(4, lb + (KW - 1) * (rs0 + (D == 3 ? rs1 : 0) + 1), Rtot);
        if (MODE == 2) sigma = io.sched[3 * (*io.iter)];
        if (PRE) {
#pragma unroll
            for (int c = 0; c < IP_CH; ++c) {
                if (c < cc) {
                    const size_t os = (size_t)(c0 + c) * geo.M + s;
                    yv[c] = ldc<T>((const T*)io.ys, os);
                    pv[c] = io.ps[os];
                    uv[c] = io.u[os];
                }
            }
        }
    }
    if (!mbar_wait_bounded(&bar, 0, io.wait)) {
        if (io.flag) atomicExch(io.flag, 1);
        mbar_wait_bounded(&bar, 0, KP_DRAIN_CYCLES);      // copies still in flight land in this CTA's memory
        return;
    }
    if (!act) return;
    // all coils of the group tap by tap: each tap's weight is formed once (no table of 64 weight
    // products held across coils); each coil's sum runs over the taps in the same order
    float2 accs[IP_CH];
#pragma unroll
    for (int c = 0; c < IP_CH; ++c) accs[c] = make_float2(0.f, 0.f);
    const float2* base = sg + lb;
#pragma unroll
    for (int a = 0; a < KW; ++a)
#pragma unroll
        for (int b = 0; b < KW; ++b) {
            const float wab = w[0][a] * w[1][b];
#pragma unroll
            for (int e = 0; e < (D == 2 ? 1 : KW); ++e) {
                const float ww = D == 2 ? wab : wab * w[D - 1][e];
                const int off = D == 2 ? a * rs0 + b : a * rs0 + b * rs1 + e;
#pragma unroll
                for (int c = 0; c < IP_CH; ++c) {
                    if (c < cc) {
                        const float2 v = base[c * Rtot + off];
                        accs[c].x = fmaf(ww, v.x, accs[c].x);
                        accs[c].y = fmaf(ww, v.y, accs[c].y);
                    }
                }
            }
        }
#pragma unroll
    for (int c = 0; c < IP_CH; ++c) {
        if (c >= cc) break;
        float2 acc = accs[c];
        acc.x *= geo.rsqrtN;
        acc.y *= geo.rsqrtN;
        const size_t os = (size_t)(c0 + c) * geo.M + s;
        if (MODE == 0) {
            const int64_t oi = io.perm ? io.perm[s] : s;
            if (KP_INB(5, oi, geo.M)) stc<T>((T*)io.out, (size_t)(c0 + c) * geo.M + oi, acc);
        } else if (MODE == 1) {
            float sc = io.ps ? io.ps[os] : 1.f;
            if (io.n2) {   // float reciprocal square root: fp64 division here costs more than the taps
                const float q = (float)*io.n2;
                sc *= q > 0.f ? rsqrtf(q) : 0.f;
            }
            io.outs[os] = make_float2(acc.x * sc, acc.y * sc);
        } else {
            // PDHG dual step (Sec. 4.1): u <- (u + sigma p (A xbar - y)) / (1 + sigma p)
            const float2 y = PRE ? yv[PRE ? c : 0] : ldc<T>((const T*)io.ys, os);
            const float sp = sigma * (PRE ? pv[PRE ? c : 0] : io.ps[os]);
            const float inv = 1.f / (1.f + sp);
            const float2 uo = PRE ? uv[PRE ? c : 0] : io.u[os];
            io.u[os] = make_float2((uo.x + sp * (acc.x - y.x)) * inv, (uo.y + sp * (acc.y - y.y)) * inv);
        }
    }
}

template <int D, int MODE, typename T>
__global__ void __launch_bounds__(IP_THREADS, 4)
k_interp_tile(const int4* __restrict__ items, const int* __restrict__ k0t, const float* __restrict__ wt,
              const float2* __restrict__ grid, Geom geo, Tiles tl, InterpIO io) {
    interp_tile_body<D, MODE, T>(items, k0t, wt, grid, geo, tl, io, blockIdx.x, blockIdx.y);
}

// The same over the cases of a batch: block b belongs to the case c with boff[c] <= b <
// boff[c + 1]; within it, item (b - boff[c]) mod n_items of coil group (b - boff[c]) / n_items.
template <int D, int MODE, typename T>
__global__ void __launch_bounds__(IP_THREADS, 4)
k_interp_tile_b(const BInterp* __restrict__ cs, const int* __restrict__ boff, int ncase) {
    const int c = batch_case(boff, ncase, (int)blockIdx.x);
    const BInterp& a = cs[c];
    const int lb = (int)blockIdx.x - boff[c];
    interp_tile_body<D, MODE, T>(a.items, a.k0t, a.wt, a.grid, a.geo, a.tl, a.io, lb % a.nx, lb / a.nx);
}

// ---------------------------------------------------------------- adjoint: spread
// One CTA per (spreading work item, group of CH coils), NW warps.  The item's samples (their
// coil values, first taps and weights) are staged in shared memory SP_CHUNK at a time by all
// threads; then each warp takes one sample at a time, its lanes covering distinct (tap, coil)
// pairs, and adds into its own private copy of the tile, so no atomics are needed.  The
// private copies are summed and the tile is stored (or, for a tile split over several items,
// added with global atomics into a region cleared beforehand).  Tile coordinates are shifted
// (Tiles::sh).  CH and NW trade occupancy (smaller copies, more warps per SM) against work
// repeated per coil group (staging and tap decoding); the autotuner picks.
constexpr int SP_CHUNK = 256;      // samples staged at a time (and the interpolation item size)

// Shared-memory layout of one private tile copy (one coil, re and im planes), for the largest
// tile edge (16 in 2D, 8 in 3D).  Strides are padded so that the 32 lanes of a warp hit 32
// different banks.
template <int D> struct SpL;
template <> struct SpL<2> {
    // lanes (ta, tb, coil parity h): 20 ta + tb + 2 PLANE h covers 32 distinct banks
    static constexpr int TS = 16, PLANE = 328;
    __device__ static constexpr int stride(int d) { return d == 0 ? 20 : 1; }
};
template <> struct SpL<3> {
    // (la, lb, lc) -> 68 la + 8 lb + lc: for 4 consecutive lb, 4 consecutive lc and two
    // consecutive la the banks (4 la + 8 lb + lc) mod 32 are all distinct
    static constexpr int TS = 8, PLANE = 544;
    __device__ static constexpr int stride(int d) { return d == 0 ? 68 : (d == 1 ? 8 : 1); }
};

template <int D, int CH, int NW>
static size_t spread_smem() {
    return (size_t)NW * CH * 2 * (D == 2 ? SpL<2>::PLANE : SpL<3>::PLANE) * sizeof(float) +
           (size_t)SP_CHUNK * (CH * sizeof(float2) + D * KW * sizeof(float) + D * sizeof(int));
}

template <int D, typename UT, int CH, int NW>
__global__ void __launch_bounds__(NW * 32)
k_spread(const int* __restrict__ k0t, const float* __restrict__ wt, const UT* __restrict__ u,
         const int* __restrict__ perm, const int* __restrict__ ext, const int4* __restrict__ items, Geom geo,
         Tiles tl, float2* __restrict__ grid) {
    using LY = SpL<D>;
    static_assert(D == 3 || CH % 2 == 0 || CH == 1, "2D lanes split coils by parity");
    extern __shared__ float smem[];
    float* acc = smem;                                              // [NW][CH][2][PLANE]
    float2* su = (float2*)(acc + NW * CH * 2 * LY::PLANE);          // [SP_CHUNK][CH]
    float* sw = (float*)(su + SP_CHUNK * CH);                       // [SP_CHUNK][D][KW]
    unsigned* sp = (unsigned*)(sw + SP_CHUNK * D * KW);             // [SP_CHUNK][D] 4 packed int8 tap coordinates
    const int4 it = items[blockIdx.x];
    const int tile = it.x, beg = it.y, end = it.z;
    const bool split = it.w >= 0;
    const int c0 = blockIdx.y * CH;
    const int cc = min(CH, geo.C - c0);
    int o[MAXD], e[MAXD];
    {
        int r = tile;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            const int tc = r % tl.nt[d];
            r /= tl.nt[d];
            o[d] = tc * tl.ts[d];
            e[d] = min(tl.ts[d], geo.g[d] - o[d]);
        }
    }
    {
        float4* a4 = (float4*)acc;
        for (int i = threadIdx.x; i < NW * CH * 2 * LY::PLANE / 4; i += blockDim.x) a4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* my = acc + warp * CH * 2 * LY::PLANE;
    for (int sb = beg; sb < end; sb += SP_CHUNK) {
        const int n = min(SP_CHUNK, end - sb);
        __syncthreads();
        // stage the samples: coil values, weights, and the local coordinate of every tap
        // inside this tile (-1 where the tap falls outside)
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int s = ext[sb + i];
            const int64_t un = perm ? perm[s] : s;
#pragma unroll
            for (int c = 0; c < CH; ++c)
                su[i * CH + c] = c < cc ? ldc<UT>(u, (size_t)(c0 + c) * geo.M + un) : make_float2(0.f, 0.f);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const int p0 = tshift(k0t[(int64_t)d * geo.M + s], tl.sh[d], geo.g[d]);
                unsigned pk = 0;
#pragma unroll
                for (int j = 0; j < KW; ++j) {
                    int pp = p0 + j;
                    if (pp >= geo.g[d]) pp -= geo.g[d];
                    const int l = pp - o[d];
                    const unsigned byte = (l >= 0 && l < e[d]) ? (unsigned)l : 0xFFu;
                    pk |= byte << (8 * j);
                    sw[(i * D + d) * KW + j] = wt[(int64_t)(d * KW + j) * geo.M + s];
                }
                sp[i * D + d] = pk;
            }
        }
        __syncthreads();
        // Each lane's updates of one sample are independent read-modify-writes of its warp's
        // private copy: all loads are issued before any store.
        if (D == 2) {
            // lanes: taps (ta, tb) x coil parity h; coils h, h + 2, ... (CH = 1: h = 1 idle)
            constexpr int CL = CH == 1 ? 1 : CH / 2;   // coils per lane
            const int ta = (lane >> 2) & 3, tb = lane & 3, h = lane >> 4;
            const bool lane_on = CH > 1 || h == 0;
            for (int i = warp; i < n; i += NW) {
                const int la = (int)(signed char)(sp[i * D] >> (8 * ta));
                const int lb = (int)(signed char)(sp[i * D + 1] >> (8 * tb));
                const bool ok = lane_on && la >= 0 && lb >= 0;
                const int lo = la * LY::stride(0) + lb;
                const float w = sw[(i * D) * KW + ta] * sw[(i * D + 1) * KW + tb];
                float rr[CL], ii[CL];
                float2 uv[CL];
#pragma unroll
                for (int k = 0; k < CL; ++k) {
                    const int c = CH == 1 ? 0 : h + 2 * k;
                    uv[k] = su[i * CH + c];
                    if (ok) { float* pl = my + c * 2 * LY::PLANE; rr[k] = pl[lo]; ii[k] = pl[LY::PLANE + lo]; }
                }
#pragma unroll
                for (int k = 0; k < CL; ++k) {
                    const int c = CH == 1 ? 0 : h + 2 * k;
                    if (ok) {
                        float* pl = my + c * 2 * LY::PLANE;
                        pl[lo] = fmaf(w, uv[k].x, rr[k]);
                        pl[LY::PLANE + lo] = fmaf(w, uv[k].y, ii[k]);
                    }
                }
                __syncwarp();
            }
        } else {
            const int tb = (lane >> 2) & 3, tc = lane & 3, ta0 = lane >> 4;   // taps (ta0 + 2k, tb, tc), k = 0, 1
            for (int i = warp; i < n; i += NW) {
                const int lb = (int)(signed char)(sp[i * D + 1] >> (8 * tb));
                const int lc = (int)(signed char)(sp[i * D + 2] >> (8 * tc));
                const float wbc = sw[(i * D + 1) * KW + tb] * sw[(i * D + 2) * KW + tc];
                const int laA = (int)(signed char)(sp[i * D] >> (8 * ta0));
                const int laB = (int)(signed char)(sp[i * D] >> (8 * (ta0 + 2)));
                const bool okA = laA >= 0 && lb >= 0 && lc >= 0, okB = laB >= 0 && lb >= 0 && lc >= 0;
                const int loA = laA * LY::stride(0) + lb * LY::stride(1 % D) + lc;
                const int loB = laB * LY::stride(0) + lb * LY::stride(1 % D) + lc;
                const float wA = sw[(i * D) * KW + ta0] * wbc, wB = sw[(i * D) * KW + ta0 + 2] * wbc;
                float rA[CH], iA[CH], rB[CH], iB[CH];
                float2 uv[CH];
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    uv[c] = su[i * CH + c];
                    float* pl = my + c * 2 * LY::PLANE;
                    if (okA) { rA[c] = pl[loA]; iA[c] = pl[LY::PLANE + loA]; }
                    if (okB) { rB[c] = pl[loB]; iB[c] = pl[LY::PLANE + loB]; }
                }
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    float* pl = my + c * 2 * LY::PLANE;
                    if (okA) { pl[loA] = fmaf(wA, uv[c].x, rA[c]); pl[LY::PLANE + loA] = fmaf(wA, uv[c].y, iA[c]); }
                    if (okB) { pl[loB] = fmaf(wB, uv[c].x, rB[c]); pl[LY::PLANE + loB] = fmaf(wB, uv[c].y, iB[c]); }
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    int P = 1;
#pragma unroll
    for (int d = 0; d < D; ++d) P *= tl.ts[d];
    for (int i = threadIdx.x; i < cc * P; i += blockDim.x) {
        const int c = i / P;
        int r = i - c * P;
        int lidx[MAXD];
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { lidx[d] = r % tl.ts[d]; r /= tl.ts[d]; }
        bool in = true;
        int lo = 0;
        int64_t gflat = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            if (lidx[d] >= e[d]) in = false;
            lo += lidx[d] * LY::stride(d);
            gflat = gflat * geo.g[d] + tunshift(o[d] + lidx[d], tl.sh[d], geo.g[d]);
        }
        if (!in) continue;
        float2 v = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const float* pl = acc + (w * CH + c) * 2 * LY::PLANE;
            v.x += pl[lo];
            v.y += pl[LY::PLANE + lo];
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

// Variant with interleaved complex storage: each warp's private tile copy holds, per grid
// point, the 4 coils of the CTA's group as two float4 (coil pairs), so a tap is one 128-bit
// load, four FMAs and one 128-bit store for two coils.  Rows are padded to 16 (mod 128) bytes
// so that the 8 lanes of each quarter-warp (two rows x four consecutive points) fall on
// distinct banks.  2D lanes: (coil pair, ta, tb); 3D lanes: (ta0, tb, tc), two taps and both
// coil pairs each.
template <int D> struct SpV;
template <> struct SpV<2> {
    static constexpr int ROW = 33;                 // float4 per row: 16 points x 2 pairs + 1 pad
    static constexpr int COPY = 16 * ROW;          // float4 per private copy
    __device__ static int idx(int l0, int l1, int, int k) { return l0 * ROW + l1 * 2 + k; }
};
template <> struct SpV<3> {
    static constexpr int ROW = 17;                 // 8 points x 2 pairs + 1 pad
    static constexpr int PLANE = 8 * ROW;
    static constexpr int COPY = 8 * PLANE;
    __device__ static int idx(int l0, int l1, int l2, int k) { return l0 * PLANE + l1 * ROW + l2 * 2 + k; }
};

template <int D, int NW>
static size_t spread_v_smem() {
    return (size_t)NW * SpV<D>::COPY * sizeof(float4) +
           (size_t)SP_CHUNK * (4 * sizeof(float2) + D * KW * sizeof(float) + D * sizeof(int));
}

template <int D, typename UT, int NW>
__device__ __forceinline__ void spread_v_body(const int* __restrict__ k0t, const float* __restrict__ wt,
                                              const UT* __restrict__ u, const int* __restrict__ perm,
                                              const int* __restrict__ ext, const int4* __restrict__ items,
                                              const Geom& geo, const Tiles& tl, float2* __restrict__ grid, int bx,
                                              int by) {
    using LV = SpV<D>;
    extern __shared__ __align__(16) float4 smv[];
    float4* acc = smv;                                              // [NW][COPY]
    float4* su4 = acc + NW * LV::COPY;                              // [SP_CHUNK][2] coil pairs
    float* sw = (float*)(su4 + SP_CHUNK * 2);                       // [SP_CHUNK][D][KW]
    unsigned* sp = (unsigned*)(sw + SP_CHUNK * D * KW);             // [SP_CHUNK][D]
    const int4 it = items[bx];
    const int tile = it.x, beg = it.y, end = it.z;
    const bool split = it.w >= 0;
    const int c0 = by * 4;
    const int cc = min(4, geo.C - c0);
    int o[MAXD], e[MAXD];
    {
        int r = tile;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            const int tc = r % tl.nt[d];
            r /= tl.nt[d];
            o[d] = tc * tl.ts[d];
            e[d] = min(tl.ts[d], geo.g[d] - o[d]);
        }
    }
    for (int i = threadIdx.x; i < NW * LV::COPY; i += blockDim.x) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4* my = acc + warp * LV::COPY;
    for (int sb = beg; sb < end; sb += SP_CHUNK) {
        const int n = min(SP_CHUNK, end - sb);
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            int s = ext[sb + i];
            bool ok = KP_INB(10, s, geo.M);
            if (!ok) s = 0;                                   // (checked build: adds zeros)
            const int64_t un = perm ? perm[s] : s;
            ok = ok && KP_INB(10, un, geo.M);
            float2 uc[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) uc[c] = ok && c < cc ? ldc<UT>(u, (size_t)(c0 + c) * geo.M + un) : make_float2(0.f, 0.f);
            su4[i * 2] = make_float4(uc[0].x, uc[0].y, uc[1].x, uc[1].y);
            su4[i * 2 + 1] = make_float4(uc[2].x, uc[2].y, uc[3].x, uc[3].y);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const int p0 = tshift(k0t[(int64_t)d * geo.M + s], tl.sh[d], geo.g[d]);
                unsigned pk = 0;
#pragma unroll
                for (int j = 0; j < KW; ++j) {
                    int pp = p0 + j;
                    if (pp >= geo.g[d]) pp -= geo.g[d];
                    const int l = pp - o[d];
                    const unsigned byte = (l >= 0 && l < e[d]) ? (unsigned)l : 0xFFu;
                    pk |= byte << (8 * j);
                    sw[(i * D + d) * KW + j] = wt[(int64_t)(d * KW + j) * geo.M + s];
                }
                sp[i * D + d] = pk;
            }
        }
        __syncthreads();
        if (D == 2) {
            const int k = lane >> 4, ta = (lane >> 2) & 3, tb = lane & 3;
            for (int i = warp; i < n; i += NW) {
                const int la = (int)(signed char)(sp[i * D] >> (8 * ta));
                const int lb = (int)(signed char)(sp[i * D + 1] >> (8 * tb));
                if (la >= 0 && lb >= 0) {
                    const float w = sw[(i * D) * KW + ta] * sw[(i * D + 1) * KW + tb];
                    const float4 uv = su4[i * 2 + k];
                    float4* a = my + LV::idx(la, lb, 0, k);
                    float4 v = *a;
                    v.x = fmaf(w, uv.x, v.x); v.y = fmaf(w, uv.y, v.y);
                    v.z = fmaf(w, uv.z, v.z); v.w = fmaf(w, uv.w, v.w);
                    *a = v;
                }
                __syncwarp();
            }
        } else {
            const int ta0 = lane >> 4, tb = (lane >> 2) & 3, tc = lane & 3;   // taps (ta0 + 2m, tb, tc)
            for (int i = warp; i < n; i += NW) {
                const int lb = (int)(signed char)(sp[i * D + 1] >> (8 * tb));
                const int lc = (int)(signed char)(sp[i * D + 2] >> (8 * tc));
                const int laA = (int)(signed char)(sp[i * D] >> (8 * ta0));
                const int laB = (int)(signed char)(sp[i * D] >> (8 * (ta0 + 2)));
                const bool inbc = lb >= 0 && lc >= 0;
                const bool okA = inbc && laA >= 0, okB = inbc && laB >= 0;
                if (okA || okB) {
                    const float wbc = sw[(i * D + 1) * KW + tb] * sw[(i * D + 2) * KW + tc];
                    const float wA = sw[(i * D) * KW + ta0] * wbc, wB = sw[(i * D) * KW + ta0 + 2] * wbc;
                    const float4 u0 = su4[i * 2], u1 = su4[i * 2 + 1];
                    float4* aA = my + LV::idx(okA ? laA : 0, lb, lc, 0);
                    float4* aB = my + LV::idx(okB ? laB : 0, lb, lc, 0);
                    float4 vA0, vA1, vB0, vB1;
                    if (okA) { vA0 = aA[0]; vA1 = aA[1]; }
                    if (okB) { vB0 = aB[0]; vB1 = aB[1]; }
                    if (okA) {
                        vA0.x = fmaf(wA, u0.x, vA0.x); vA0.y = fmaf(wA, u0.y, vA0.y);
                        vA0.z = fmaf(wA, u0.z, vA0.z); vA0.w = fmaf(wA, u0.w, vA0.w);
                        vA1.x = fmaf(wA, u1.x, vA1.x); vA1.y = fmaf(wA, u1.y, vA1.y);
                        vA1.z = fmaf(wA, u1.z, vA1.z); vA1.w = fmaf(wA, u1.w, vA1.w);
                        aA[0] = vA0; aA[1] = vA1;
                    }
                    if (okB) {
                        vB0.x = fmaf(wB, u0.x, vB0.x); vB0.y = fmaf(wB, u0.y, vB0.y);
                        vB0.z = fmaf(wB, u0.z, vB0.z); vB0.w = fmaf(wB, u0.w, vB0.w);
                        vB1.x = fmaf(wB, u1.x, vB1.x); vB1.y = fmaf(wB, u1.y, vB1.y);
                        vB1.z = fmaf(wB, u1.z, vB1.z); vB1.w = fmaf(wB, u1.w, vB1.w);
                        aB[0] = vB0; aB[1] = vB1;
                    }
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    // sum the private copies; one thread per (point, coil pair)
    int P = 1;
#pragma unroll
    for (int d = 0; d < D; ++d) P *= tl.ts[d];
    const int npair = (cc + 1) / 2;
    for (int i = threadIdx.x; i < npair * P; i += blockDim.x) {
        const int k = i / P;
        int r = i - k * P;
        int lidx[MAXD];
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { lidx[d] = r % tl.ts[d]; r /= tl.ts[d]; }
        bool in = true;
        int64_t gflat = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            if (lidx[d] >= e[d]) in = false;
            gflat = gflat * geo.g[d] + tunshift(o[d] + lidx[d], tl.sh[d], geo.g[d]);
        }
        if (!in || !KP_INB(10, (int64_t)(c0 + 2 * k + (2 * k + 1 < cc)) * geo.G + gflat, (int64_t)geo.C * geo.G)) continue;
        const int li = D == 2 ? LV::idx(lidx[0], lidx[D - 1], 0, k) : LV::idx(lidx[0], lidx[1 % D], lidx[D - 1], k);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const float4 t = acc[w * LV::COPY + li];
            v.x += t.x; v.y += t.y; v.z += t.z; v.w += t.w;
        }
        const int ca = c0 + 2 * k;
        float2* d0 = grid + (size_t)ca * geo.G + gflat;
        float2* d1 = d0 + geo.G;
        const bool has1 = 2 * k + 1 < cc;
        if (split) {
            atomicAdd(&d0->x, v.x);
            atomicAdd(&d0->y, v.y);
            if (has1) { atomicAdd(&d1->x, v.z); atomicAdd(&d1->y, v.w); }
        } else {
            *d0 = make_float2(v.x, v.y);
            if (has1) *d1 = make_float2(v.z, v.w);
        }
    }
}

template <int D, typename UT, int NW>
__global__ void __launch_bounds__(NW * 32)
k_spread_v(const int* __restrict__ k0t, const float* __restrict__ wt, const UT* __restrict__ u,
           const int* __restrict__ perm, const int* __restrict__ ext, const int4* __restrict__ items, Geom geo,
           Tiles tl, float2* __restrict__ grid) {
    spread_v_body<D, UT, NW>(k0t, wt, u, perm, ext, items, geo, tl, grid, blockIdx.x, blockIdx.y);
}

// The same over the cases of a batch (block b -> case and item as in k_interp_tile_b).
template <int D, typename UT, int NW>
__global__ void __launch_bounds__(NW * 32) k_spread_v_b(const BSpread* __restrict__ cs, const int* __restrict__ boff,
                                                        int ncase) {
    const int c = batch_case(boff, ncase, (int)blockIdx.x);
    const BSpread& a = cs[c];
    const int lb = (int)blockIdx.x - boff[c];
    spread_v_body<D, UT, NW>(a.k0t, a.wt, (const UT*)a.u, a.perm, a.ext, a.items, a.geo, a.tl, a.grid, lb % a.nx,
                             lb / a.nx);
}

// 3D variant in which warp w owns z-plane w of a single accumulator (8 warps, tile depth at
// most 8): every warp walks every staged sample and applies only the taps in its own plane
// (at most one of a sample's four z taps), so no two warps touch the same address and there
// are no private copies to clear and sum.  CG coils per CTA, stored per grid point as CG/2
// float4 coil pairs; lanes (ty, tx, h) take one (y, x) tap each and coil pairs h (CG = 4) or
// 2h, 2h + 1 (CG = 8).  For CG = 8 the pair slot is XOR-swizzled with bit 1 of x so that each
// quarter-warp (four consecutive x, two h) reads eight distinct 16-byte bank groups.
template <int CG> struct SpZ {
    static constexpr int NP = CG / 2;              // float4 per grid point
    static constexpr int COPY = 512 * NP;
    __device__ static int idx(int z, int y, int x, int k) {
        const int slot = CG == 8 ? (k ^ ((x >> 1) & 1)) : k;
        return ((z * 8 + y) * 8 + x) * NP + slot;
    }
};

template <int CG>
static size_t spread_z_smem() {
    return (size_t)SpZ<CG>::COPY * sizeof(float4) + (size_t)SP_CHUNK * (CG * sizeof(float2) + 3 * KW * sizeof(float) + 3 * sizeof(int));
}

template <typename UT, int CG>
__global__ void __launch_bounds__(256)
k_spread_z(const int* __restrict__ k0t, const float* __restrict__ wt, const UT* __restrict__ u,
           const int* __restrict__ perm, const int* __restrict__ ext, const int4* __restrict__ items, Geom geo,
           Tiles tl, float2* __restrict__ grid) {
    constexpr int D = 3, NP = CG / 2;
    using LZ = SpZ<CG>;
    extern __shared__ __align__(16) float4 smz[];
    float4* acc = smz;                                              // [8][8][8][NP]
    float4* su4 = acc + LZ::COPY;                                   // [SP_CHUNK][NP]
    float* sw = (float*)(su4 + SP_CHUNK * NP);                      // [SP_CHUNK][3][KW]
    unsigned* sp = (unsigned*)(sw + SP_CHUNK * D * KW);             // [SP_CHUNK][3]
    const int4 it = items[blockIdx.x];
    const int tile = it.x, beg = it.y, end = it.z;
    const bool split = it.w >= 0;
    const int c0 = blockIdx.y * CG;
    const int cc = min(CG, geo.C - c0);
    int o[MAXD], e[MAXD];
    {
        int r = tile;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            const int tc = r % tl.nt[d];
            r /= tl.nt[d];
            o[d] = tc * tl.ts[d];
            e[d] = min(tl.ts[d], geo.g[d] - o[d]);
        }
    }
    for (int i = threadIdx.x; i < LZ::COPY; i += blockDim.x) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ty = lane >> 3, tx = (lane >> 1) & 3, h = lane & 1;
    const unsigned wz4 = (unsigned)warp * 0x01010101u;
    for (int sb = beg; sb < end; sb += SP_CHUNK) {
        const int n = min(SP_CHUNK, end - sb);
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int s = ext[sb + i];
            const int64_t un = perm ? perm[s] : s;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const float2 ua = 2 * k < cc ? ldc<UT>(u, (size_t)(c0 + 2 * k) * geo.M + un) : make_float2(0.f, 0.f);
                const float2 ub = 2 * k + 1 < cc ? ldc<UT>(u, (size_t)(c0 + 2 * k + 1) * geo.M + un) : make_float2(0.f, 0.f);
                su4[i * NP + k] = make_float4(ua.x, ua.y, ub.x, ub.y);
            }
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const int p0 = tshift(k0t[(int64_t)d * geo.M + s], tl.sh[d], geo.g[d]);
                unsigned pk = 0;
#pragma unroll
                for (int j = 0; j < KW; ++j) {
                    int pp = p0 + j;
                    if (pp >= geo.g[d]) pp -= geo.g[d];
                    const int l = pp - o[d];
                    const unsigned byte = (l >= 0 && l < e[d]) ? (unsigned)l : 0xFFu;
                    pk |= byte << (8 * j);
                    sw[(i * D + d) * KW + j] = wt[(int64_t)(d * KW + j) * geo.M + s];
                }
                sp[i * D + d] = pk;
            }
        }
        __syncthreads();
        for (int i = 0; i < n; ++i) {
            const unsigned mz = __vcmpeq4(sp[i * D], wz4);      // which z tap lies in my plane
            if (mz == 0) continue;                              // warp-uniform
            const int jz = (__ffs((int)mz) - 1) >> 3;
            const int ly = (int)(signed char)(sp[i * D + 1] >> (8 * ty));
            const int lx = (int)(signed char)(sp[i * D + 2] >> (8 * tx));
            if (ly >= 0 && lx >= 0) {
                const float w = sw[(i * D) * KW + jz] * sw[(i * D + 1) * KW + ty] * sw[(i * D + 2) * KW + tx];
#pragma unroll
                for (int j = 0; j < NP / 2; ++j) {
                    const int k = (NP / 2) * h + j;
                    const float4 uv = su4[i * NP + k];
                    float4* a = acc + LZ::idx(warp, ly, lx, k);
                    float4 v = *a;
                    v.x = fmaf(w, uv.x, v.x); v.y = fmaf(w, uv.y, v.y);
                    v.z = fmaf(w, uv.z, v.z); v.w = fmaf(w, uv.w, v.w);
                    *a = v;
                }
            }
        }
    }
    __syncthreads();
    int P = 1;
#pragma unroll
    for (int d = 0; d < D; ++d) P *= tl.ts[d];
    const int npair = (cc + 1) / 2;
    for (int i = threadIdx.x; i < npair * P; i += blockDim.x) {
        const int k = i / P;
        int r = i - k * P;
        int lidx[MAXD];
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { lidx[d] = r % tl.ts[d]; r /= tl.ts[d]; }
        bool in = true;
        int64_t gflat = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            if (lidx[d] >= e[d]) in = false;
            gflat = gflat * geo.g[d] + tunshift(o[d] + lidx[d], tl.sh[d], geo.g[d]);
        }
        if (!in) continue;
        const float4 v = acc[LZ::idx(lidx[0], lidx[1], lidx[2], k)];
        const int ca = c0 + 2 * k;
        float2* d0 = grid + (size_t)ca * geo.G + gflat;
        float2* d1 = d0 + geo.G;
        const bool has1 = 2 * k + 1 < cc;
        if (split) {
            atomicAdd(&d0->x, v.x);
            atomicAdd(&d0->y, v.y);
            if (has1) { atomicAdd(&d1->x, v.z); atomicAdd(&d1->y, v.w); }
        } else {
            *d0 = make_float2(v.x, v.y);
            if (has1) *d1 = make_float2(v.z, v.w);
        }
    }
}

// Two-phase 3D spreading (variants 10, 11).  Phase A: one CTA per own-sample item (samples
// whose first tap lies in the tile, contiguous in sorted order, which within a tile is ordered
// by that first tap) accumulates every tap of each sample once into a padded tile of
// (8 + W - 1)^3 points in shared memory (no tap falls outside it) and writes the padded tile
// to its slot.  The CTA has 2 NP warps for NP coil pairs: warp w owns coil pair w mod NP and the
// padded z-planes of parity w / NP, so for each sample every warp updates its two planes x
// 16 (y, x) taps of its pair, one tap per lane, and no two warps ever write the same word.
// Consecutive samples with the same first tap have the same footprint: a lane sums their
// contributions in registers and updates shared memory once per run.  Phase B: one CTA per tile
// stores every grid point as the sum of its tile's slots and, for points within W - 1 of a low
// face, of the lower neighbours' halos (periodic): no atomics, no clearing, fixed sum order.
constexpr int PT = 8 + KW - 1;                 // padded tile edge
constexpr int OT_RS = 12;                      // float4 per padded row: x padded to 12 so that a quarter-warp's
constexpr int OT_PS = PT * OT_RS;              // lanes (4 consecutive x, 2 rows) hit 8 different bank groups
constexpr int OT_PAIR = PT * OT_PS;            // float4 per coil pair
constexpr int OT_CHUNK = 128;                  // samples staged at a time
// slot layout of a padded tile per coil: rows of SL_RS points (x padded from 11 to 12, so a row
// is 96 bytes and the 8 points a gather warp reads from it sit in two aligned 32-byte sectors)
constexpr int SL_RS = 12, SL_PS = PT * SL_RS, SL_P = PT * SL_PS;

template <int NP>
static size_t spread_own_smem() {
    // accumulator + per staged sample (one sentinel slot more): NP coil pairs, the y x weight
    // products, and per warp parity the plane offset and the two z weights
    return (size_t)NP * OT_PAIR * sizeof(float4) +
           (size_t)(OT_CHUNK + 1) * (NP * sizeof(float4) + KW * KW * sizeof(float) + 2 * sizeof(int) + 4 * sizeof(float));
}

// Phase A: one CTA per own-sample item (the samples whose first tap lies in one tile, at most
// OT_CHUNK at a time) and group of 2 NP coils.  Warp (pair, par) owns coil pair `pair` and the
// padded z-planes of parity `par`; its 32 lanes are the (z, y, x) taps (jsel: the 2 z taps of
// that parity, yx: the 16 (y, x) taps).  Staging computes per sample and parity the plane
// offset of the first tap of that parity and the two z weights, so the inner loop only reads
// them; consecutive samples with the same offset (same planes, rows and columns: a run) are
// summed in registers and added to the accumulator once.
template <typename UT, int NP>
__global__ void __launch_bounds__(NP * 64)
k_spread_own(const int* __restrict__ k0t, const float* __restrict__ wt, const UT* __restrict__ u,
             const int* __restrict__ perm, const int4* __restrict__ items, Geom geo, Tiles tl,
             float2* __restrict__ halo) {
    constexpr int D = 3, NT = NP * 64, CH = OT_CHUNK + 1;
    extern __shared__ __align__(16) float4 smo[];
    float4* acc = smo;                                              // [NP][PT][PT][OT_RS]
    float4* su = acc + NP * OT_PAIR;                                // [CH][NP] coil pairs
    float* swyx = (float*)(su + CH * NP);                           // [CH][KW * KW] y x weight products
    int* soff = (int*)(swyx + CH * KW * KW);                        // [2][CH] plane offset per parity
    float* swz = (float*)(soff + 2 * CH);                           // [2][CH][2] z weights per parity
    const int4 it = items[blockIdx.x];
    const int tile = it.x, beg = it.y, end = it.z, slot = it.w;
    const int c0 = blockIdx.y * 2 * NP;
    const int cc = min(2 * NP, geo.C - c0);
    int o[MAXD];
    {
        int r = tile;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            const int tc = r % tl.nt[d];
            r /= tl.nt[d];
            o[d] = tc * tl.ts[d];
        }
    }
    for (int i = threadIdx.x; i < NP * OT_PAIR; i += NT) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pair = warp % NP, par = warp / NP;
    const int jsel = lane >> 4, yx = lane & 15;
    // this lane's tap relative to the first tap of the warp's parity: z + 2 jsel, y = yx >> 2, x = yx & 3
    float4* const mine = acc + pair * OT_PAIR + 2 * jsel * OT_PS + (yx >> 2) * OT_RS + (yx & 3);
    const int* const offs = soff + par * CH;
    const float* const wzs = swz + par * CH * 2 + jsel;
    const bool live = 2 * pair < cc;
    for (int s0 = beg; s0 < end; s0 += OT_CHUNK) {
        const int n = min(OT_CHUNK, end - s0);
        __syncthreads();
        for (int i = threadIdx.x; i <= n; i += NT) {
            if (i == n) {                                           // sentinel: read by the last prefetch only
                soff[i] = soff[CH + i] = -1;
                continue;
            }
            const int s = s0 + i;
            const int64_t un = perm ? perm[s] : s;
            int l[D];
            bool ok = KP_INB(6, un, geo.M);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                l[d] = tshift(k0t[(int64_t)d * geo.M + s], tl.sh[d], geo.g[d]) - o[d];   // in [0, ts)
                if (!KP_INB(7, l[d], tl.ts[d])) { ok = false; l[d] = 0; }   // (checked build: adds zeros)
            }
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const float2 ua = ok && 2 * k < cc ? ldc<UT>(u, (size_t)(c0 + 2 * k) * geo.M + un) : make_float2(0.f, 0.f);
                const float2 ub = ok && 2 * k + 1 < cc ? ldc<UT>(u, (size_t)(c0 + 2 * k + 1) * geo.M + un) : make_float2(0.f, 0.f);
                su[i * NP + k] = make_float4(ua.x, ua.y, ub.x, ub.y);
            }
            float wz[KW], wy[KW], wx[KW];
#pragma unroll
            for (int j = 0; j < KW; ++j) {
                wz[j] = wt[(int64_t)j * geo.M + s];
                wy[j] = wt[(int64_t)(KW + j) * geo.M + s];
                wx[j] = wt[(int64_t)(2 * KW + j) * geo.M + s];
            }
#pragma unroll
            for (int a = 0; a < KW; ++a)
#pragma unroll
                for (int b = 0; b < KW; ++b) swyx[i * KW * KW + a * KW + b] = wy[a] * wx[b];
            // parity q: the first z tap of that parity is jz0 = (q ^ l0) & 1, its plane l0 + jz0
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int jz0 = (q ^ l[0]) & 1;
                soff[q * CH + i] = (l[0] + jz0) * OT_PS + l[1] * OT_RS + l[2];
                swz[(q * CH + i) * 2] = wz[jz0];
                swz[(q * CH + i) * 2 + 1] = wz[jz0 + 2];
            }
        }
        __syncthreads();
        if (live && n > 0) {
            int run = -1;                                            // current run's offset, warp-uniform
            float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
            // sample i's staged values are in registers before its turn (the sentinel makes the
            // prefetch of sample n harmless)
            int off = offs[0];
            float wz = wzs[0], wyx = swyx[yx];
            float4 uv = su[pair];
            for (int i = 0; i < n; ++i) {
                const int oi = off;
                const float w = wz * wyx;
                const float4 ui = uv;
                off = offs[i + 1];
                wz = wzs[(i + 1) * 2];
                wyx = swyx[(i + 1) * KW * KW + yx];
                uv = su[(i + 1) * NP + pair];
                if (oi != run) {
                    if (run >= 0) {
                        float4 v = mine[run];
                        v.x += r.x; v.y += r.y; v.z += r.z; v.w += r.w;
                        mine[run] = v;
                    }
                    run = oi;
                    r = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                r.x = fmaf(w, ui.x, r.x); r.y = fmaf(w, ui.y, r.y);
                r.z = fmaf(w, ui.z, r.z); r.w = fmaf(w, ui.w, r.w);
            }
            if (run >= 0) {
                float4 v = mine[run];
                v.x += r.x; v.y += r.y; v.z += r.z; v.w += r.w;
                mine[run] = v;
            }
        }
    }
    __syncthreads();
    // padded tile -> slot, coil-major: halo[(slot * C + c) * SL_P + (z * PT + y) * SL_RS + x]
    // (the accumulator rows have the slot's row length, so the copy is row for row)
    static_assert(OT_RS == SL_RS, "accumulator and slot rows have the same length");
    const int npair = (cc + 1) / 2;
    if (!KP_INB(7, slot, gridDim.x)) return;                       // one slot per item
    for (int i = threadIdx.x; i < npair * SL_P; i += NT) {
        const int k = i / SL_P, pt = i - k * SL_P;
        if (pt % SL_RS >= PT) continue;                             // the row's padding point
        const float4 v = acc[k * OT_PAIR + pt];
        float2* d0 = halo + ((size_t)slot * geo.C + c0 + 2 * k) * SL_P + pt;
        *d0 = make_float2(v.x, v.y);
        if (2 * k + 1 < cc) d0[SL_P] = make_float2(v.z, v.w);
    }
}

// Phase B: one CTA per tile (empty tiles included, so every grid point is stored once).  The
// tile's value is the sum of its own slots' 8^3 cores and of the halos that its 7 lower
// neighbours (periodic) spill into it: the neighbour across axis set m covers the sub-box with
// extent KW - 1 along the axes in m and the full tile along the others, read from the
// neighbour's slots at the padded offset where its core ends.  Coils go GB_CB at a time, all
// of a chunk at once (a slot holds its coils contiguously), so every pass issues independent
// loads for GB_CB x 512 (point, coil) pairs and the CTA meets at one barrier per pass, not per
// coil: the own cores into registers (16 pairs per thread), then one pass per non-empty
// neighbour into the shared accumulator, then the chunk is stored.  Every slot point is read
// once; offsets come from per-CTA tables.
constexpr int GB_CB = 8;                       // coils per chunk (the accumulator holds GB_CB x 512 points)
constexpr int GB_T = 256;                      // threads
constexpr int GB_PER = GB_CB * 512 / GB_T;     // (point, coil) pairs per thread in the own pass

__global__ void __launch_bounds__(GB_T)
k_halo_gather(const float2* __restrict__ halo, const int* __restrict__ tslot, Geom geo, Tiles tl,
              float2* __restrict__ grid) {
    __shared__ float2 acc[GB_CB * 512];
    __shared__ int nb_beg[8], nb_end[8], nb_off[8];
    __shared__ int64_t rowoff[64];     // grid offset (coil 0) of local row (lz, ly); -1 outside the grid
    __shared__ int colg[8];            // grid x of local x; -1 outside the grid
    const int tile = blockIdx.x;
    const int nt0 = tl.nt[0], nt1 = tl.nt[1], nt2 = tl.nt[2];
    const int t2 = tile % nt2, t1 = (tile / nt2) % nt1, t0 = tile / (nt2 * nt1);
    if (threadIdx.x < 8) {
        const int m = threadIdx.x;
        const int ts0 = tl.ts[0], ts1 = tl.ts[1], ts2 = tl.ts[2];
        const int b0 = (m >> 2) & 1, b1 = (m >> 1) & 1, b2 = m & 1;
        const int n0 = b0 ? (t0 == 0 ? nt0 - 1 : t0 - 1) : t0;
        const int n1 = b1 ? (t1 == 0 ? nt1 - 1 : t1 - 1) : t1;
        const int n2 = b2 ? (t2 == 0 ? nt2 - 1 : t2 - 1) : t2;
        const int nb = (n0 * nt1 + n1) * nt2 + n2;
        nb_beg[m] = tslot[nb];
        nb_end[m] = tslot[nb + 1];
        // (checked build: a slot range beyond the slots the own phase wrote is skipped)
        if (nb_end[m] > nb_beg[m] && !(KP_INB(8, nb_beg[m], tslot[tl.ntiles]) && KP_INB(8, nb_end[m] - 1, tslot[tl.ntiles])))
            nb_end[m] = nb_beg[m];
        nb_off[m] = (b0 ? min(ts0, geo.g[0] - n0 * ts0) * SL_PS : 0) + (b1 ? min(ts1, geo.g[1] - n1 * ts1) * SL_RS : 0) +
                    (b2 ? min(ts2, geo.g[2] - n2 * ts2) : 0);
    } else if (threadIdx.x < 8 + 64) {
        const int r = threadIdx.x - 8, lz = r >> 3, ly = r & 7;
        const int pz = t0 * tl.ts[0] + lz, py = t1 * tl.ts[1] + ly;
        rowoff[r] = (lz < min(tl.ts[0], geo.g[0] - t0 * tl.ts[0]) && ly < min(tl.ts[1], geo.g[1] - t1 * tl.ts[1]))
                        ? ((int64_t)tunshift(pz, tl.sh[0], geo.g[0]) * geo.g[1] + tunshift(py, tl.sh[1], geo.g[1])) * geo.g[2]
                        : (int64_t)-1;
    } else if (threadIdx.x < 8 + 64 + 8) {
        const int lx = threadIdx.x - 72, px = t2 * tl.ts[2] + lx;
        colg[lx] = lx < min(tl.ts[2], geo.g[2] - t2 * tl.ts[2]) ? tunshift(px, tl.sh[2], geo.g[2]) : -1;
    }
    __syncthreads();
    const int64_t sstride = (int64_t)geo.C * SL_P;       // one slot: all coils
    const int own_b = nb_beg[0], own_e = nb_end[0];
    for (int c0 = 0; c0 < geo.C; c0 += GB_CB) {
        const int cc = min(GB_CB, geo.C - c0);
        const float2* hc = halo + (int64_t)c0 * SL_P;
        // own cores: pair q = threadIdx.x + GB_T j holds coil q >> 9, point q & 511
        float2 a[GB_PER];
#pragma unroll
        for (int j = 0; j < GB_PER; ++j) a[j] = make_float2(0.f, 0.f);
        for (int sl = own_b; sl < own_e; ++sl) {
            const float2* src = hc + sl * sstride;
#pragma unroll
            for (int j = 0; j < GB_PER; ++j) {
                const int q = threadIdx.x + GB_T * j, c = q >> 9, p = q & 511;
                if (c < cc) {
                    const float2 v = src[c * SL_P + ((p >> 6) * PT + ((p >> 3) & 7)) * SL_RS + (p & 7)];
                    a[j].x += v.x;
                    a[j].y += v.y;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < GB_PER; ++j) acc[threadIdx.x + GB_T * j] = a[j];
#pragma unroll 1
        for (int m = 1; m < 8; ++m) {
            const int be = nb_beg[m], en = nb_end[m];
            if (be == en) continue;                                  // block-uniform
            __syncthreads();                                         // earlier passes' adds are done
            const int d1 = (m & 2) ? KW - 1 : 8, d2 = (m & 1) ? KW - 1 : 8;
            const int d0 = (m & 4) ? KW - 1 : 8;
            const int per_c = d0 * d1 * d2, npts = per_c * cc, off = nb_off[m];
            for (int q = threadIdx.x; q < npts; q += GB_T) {
                const int c = q / per_c, r0 = q - c * per_c;
                const int lx = r0 % d2, r = r0 / d2, ly = r % d1, lz = r / d1;
                const float2* src = hc + c * SL_P + off + (lz * PT + ly) * SL_RS + lx;
                float2 sm = make_float2(0.f, 0.f);
                for (int k = be; k < en; ++k) {
                    const float2 v = src[k * sstride];
                    sm.x += v.x;
                    sm.y += v.y;
                }
                float2& t = acc[c * 512 + (lz * 8 + ly) * 8 + lx];
                t.x += sm.x;
                t.y += sm.y;
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < cc * 512; q += GB_T) {
            const int c = q >> 9, p = q & 511;
            const int64_t ro = rowoff[p >> 3];
            const int gx = colg[p & 7];
            if (ro >= 0 && gx >= 0 && KP_INB(9, (int64_t)(c0 + c) * geo.G + ro + gx, (int64_t)geo.C * geo.G))
                grid[(int64_t)(c0 + c) * geo.G + ro + gx] = acc[q];
        }
        __syncthreads();                                             // acc is rewritten by the next chunk
    }
}

__device__ __forceinline__ void tile_local(int k, int sh, int g, int ts, int& t, int& l) {
    const int p = tshift(k, sh, g);
    t = p / ts;
    l = p - t * ts;
}

// Two-phase spreading in 2D (variant 12): phase A as in 3D but with warp-private copies of the
// padded (16 + W - 1)^2 tile (4 coils as two float4 pairs per point), each warp taking its own
// samples with every lane on a tap (lanes: coil pair, ta, tb); rows padded to 16 (mod 128)
// bytes so each quarter-warp (two rows x four points) is conflict-free.  Phase B as in 3D.
constexpr int PT2 = 16 + KW - 1;
constexpr int PT2SQ = PT2 * PT2;
constexpr int OW_ROW = 2 * PT2 + 3;            // float4 per padded row (656 bytes)
constexpr int OW_COPY = PT2 * OW_ROW;

template <int NW>
static size_t spread_own2_smem() {
    return (size_t)NW * OW_COPY * sizeof(float4) + (size_t)SP_CHUNK * (2 * sizeof(float4) + 2 * KW * sizeof(float) + sizeof(int));
}

template <typename UT, int NW>
__global__ void __launch_bounds__(NW * 32)
k_spread_own2(const int* __restrict__ k0t, const float* __restrict__ wt, const UT* __restrict__ u,
              const int* __restrict__ perm, const int4* __restrict__ items, Geom geo, Tiles tl,
              float2* __restrict__ halo) {
    constexpr int D = 2;
    extern __shared__ __align__(16) float4 smo2[];
    float4* acc = smo2;                                             // [NW][PT2][OW_ROW]
    float4* su4 = acc + NW * OW_COPY;                               // [SP_CHUNK][2]
    float* sw = (float*)(su4 + SP_CHUNK * 2);                       // [SP_CHUNK][2][KW]
    unsigned* sp = (unsigned*)(sw + SP_CHUNK * D * KW);             // [SP_CHUNK] local first taps
    const int4 it = items[blockIdx.x];
    const int tile = it.x, beg = it.y, end = it.z, slot = it.w;
    const int c0 = blockIdx.y * 4;
    const int cc = min(4, geo.C - c0);
    const int o1 = (tile % tl.nt[1]) * tl.ts[1], o0 = (tile / tl.nt[1]) * tl.ts[0];
    for (int i = threadIdx.x; i < NW * OW_COPY; i += blockDim.x) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = lane >> 4, ta = (lane >> 2) & 3, tb = lane & 3;
    float4* my = acc + warp * OW_COPY;
    for (int sb = beg; sb < end; sb += SP_CHUNK) {
        const int n = min(SP_CHUNK, end - sb);
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int s = sb + i;
            const int64_t un = perm ? perm[s] : s;
            float2 uc[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) uc[c] = c < cc ? ldc<UT>(u, (size_t)(c0 + c) * geo.M + un) : make_float2(0.f, 0.f);
            su4[i * 2] = make_float4(uc[0].x, uc[0].y, uc[1].x, uc[1].y);
            su4[i * 2 + 1] = make_float4(uc[2].x, uc[2].y, uc[3].x, uc[3].y);
            const int l0 = tshift(k0t[s], tl.sh[0], geo.g[0]) - o0;
            const int l1 = tshift(k0t[(int64_t)geo.M + s], tl.sh[1], geo.g[1]) - o1;
            sp[i] = (unsigned)l0 | ((unsigned)l1 << 8);
#pragma unroll
            for (int d = 0; d < D; ++d)
#pragma unroll
                for (int j = 0; j < KW; ++j) sw[(i * D + d) * KW + j] = wt[(int64_t)(d * KW + j) * geo.M + s];
        }
        __syncthreads();
        for (int i = warp; i < n; i += NW) {
            const unsigned pk = sp[i];
            const int y = (int)(pk & 0xFFu) + ta, x = (int)((pk >> 8) & 0xFFu) + tb;
            const float w = sw[(i * D) * KW + ta] * sw[(i * D + 1) * KW + tb];
            const float4 uv = su4[i * 2 + k];
            float4* a = my + y * OW_ROW + x * 2 + k;
            float4 v = *a;
            v.x = fmaf(w, uv.x, v.x); v.y = fmaf(w, uv.y, v.y);
            v.z = fmaf(w, uv.z, v.z); v.w = fmaf(w, uv.w, v.w);
            *a = v;
            __syncwarp();
        }
    }
    __syncthreads();
    const int npair = (cc + 1) / 2;
    for (int i = threadIdx.x; i < npair * PT2SQ; i += blockDim.x) {
        const int kp = i / PT2SQ, pt = i - kp * PT2SQ;
        const int y = pt / PT2, x = pt - y * PT2;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const float4 t = acc[w * OW_COPY + y * OW_ROW + x * 2 + kp];
            v.x += t.x; v.y += t.y; v.z += t.z; v.w += t.w;
        }
        float2* d0 = halo + ((size_t)slot * geo.C + c0 + 2 * kp) * PT2SQ + pt;
        *d0 = make_float2(v.x, v.y);
        if (2 * kp + 1 < cc) d0[PT2SQ] = make_float2(v.z, v.w);
    }
}

__global__ void __launch_bounds__(256)
k_halo_gather2(const float2* __restrict__ halo, const int* __restrict__ tslot, Geom geo, Tiles tl,
               float2* __restrict__ grid) {
    const int xb = (geo.g[1] + blockDim.x - 1) / blockDim.x;
    const int row = blockIdx.x / xb, c = blockIdx.y;
    const int k1 = (blockIdx.x - row * xb) * blockDim.x + threadIdx.x;
    if (k1 >= geo.g[1]) return;
    int t[2], l[2];
    tile_local(row, tl.sh[0], geo.g[0], tl.ts[0], t[0], l[0]);
    tile_local(k1, tl.sh[1], geo.g[1], tl.ts[1], t[1], l[1]);
    int tt[2][2], ll[2][2];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        tt[d][0] = t[d];
        ll[d][0] = l[d];
        tt[d][1] = t[d] == 0 ? tl.nt[d] - 1 : t[d] - 1;
        ll[d][1] = l[d] + min(tl.ts[d], geo.g[d] - tt[d][1] * tl.ts[d]);
    }
    const size_t cstride = (size_t)geo.C * PT2SQ;
    const float2* hc = halo + (size_t)c * PT2SQ;
    float2 sum = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int b0 = m >> 1, b1 = m & 1;
        if ((b0 && l[0] >= KW - 1) || (b1 && l[1] >= KW - 1)) continue;
        const int tile = tt[0][b0] * tl.nt[1] + tt[1][b1];
        const int pt = ll[0][b0] * PT2 + ll[1][b1];
        const int s1 = tslot[tile + 1];
        for (int sl = tslot[tile]; sl < s1; ++sl) {
            const float2 v = hc[(size_t)sl * cstride + pt];
            sum.x += v.x;
            sum.y += v.y;
        }
    }
    grid[(size_t)c * geo.G + (size_t)row * geo.g[1] + k1] = sum;
}

// Variant with one shared accumulator per CTA and up to SPA_CH coils per CTA (one coil group
// for C <= 16): the tap geometry of a sample is staged once for all its coils and the lanes
// add with shared-memory atomics (a warp's lanes cover distinct (tap, coil) addresses; only
// warps working on the same point contend).
constexpr int SPA_CH = 16;
constexpr int SPA_THREADS = 256;

// cs = coils per CTA (min(C, SPA_CH)): the accumulator and the staged coil values are sized
// for the coils actually present, so few-coil plans fit several CTAs per SM
template <int D>
static size_t spread_atomic_smem(int cs) {
    return (size_t)cs * 2 * (D == 2 ? SpL<2>::PLANE : SpL<3>::PLANE) * sizeof(float) +
           (size_t)SP_CHUNK * (cs * sizeof(float2) + D * KW * sizeof(float) + D * sizeof(int));
}

template <int D, typename UT>
__global__ void __launch_bounds__(SPA_THREADS)
k_spread_atomic(const int* __restrict__ k0t, const float* __restrict__ wt, const UT* __restrict__ u,
                const int* __restrict__ perm, const int* __restrict__ ext, const int4* __restrict__ items, Geom geo,
                Tiles tl, float2* __restrict__ grid) {
    using LY = SpL<D>;
    extern __shared__ float smem[];
    const int cs = min(geo.C, SPA_CH);                              // coils per CTA (stride)
    float* acc = smem;                                              // [cs][2][PLANE]
    float2* su = (float2*)(acc + cs * 2 * LY::PLANE);               // [SP_CHUNK][cs]
    float* sw = (float*)(su + SP_CHUNK * cs);                       // [SP_CHUNK][D][KW]
    unsigned* sp = (unsigned*)(sw + SP_CHUNK * D * KW);             // [SP_CHUNK][D]
    const int4 it = items[blockIdx.x];
    const int tile = it.x, beg = it.y, end = it.z;
    const bool split = it.w >= 0;
    const int c0 = blockIdx.y * SPA_CH;
    const int cc = min(SPA_CH, geo.C - c0);
    int o[MAXD], e[MAXD];
    {
        int r = tile;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            const int tc = r % tl.nt[d];
            r /= tl.nt[d];
            o[d] = tc * tl.ts[d];
            e[d] = min(tl.ts[d], geo.g[d] - o[d]);
        }
    }
    for (int i = threadIdx.x; i < cc * 2 * LY::PLANE; i += blockDim.x) acc[i] = 0.f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int sb = beg; sb < end; sb += SP_CHUNK) {   // SP_CHUNK samples at a time
    const int n = min(SP_CHUNK, end - sb);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int s = ext[sb + i];
        const int64_t un = perm ? perm[s] : s;
        for (int c = 0; c < cc; ++c) su[i * cs + c] = ldc<UT>(u, (size_t)(c0 + c) * geo.M + un);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int p0 = tshift(k0t[(int64_t)d * geo.M + s], tl.sh[d], geo.g[d]);
            unsigned pk = 0;
#pragma unroll
            for (int j = 0; j < KW; ++j) {
                int pp = p0 + j;
                if (pp >= geo.g[d]) pp -= geo.g[d];
                const int l = pp - o[d];
                const unsigned byte = (l >= 0 && l < e[d]) ? (unsigned)l : 0xFFu;
                pk |= byte << (8 * j);
                sw[(i * D + d) * KW + j] = wt[(int64_t)(d * KW + j) * geo.M + s];
            }
            sp[i * D + d] = pk;
        }
    }
    __syncthreads();
    if (D == 2) {
        const int ta = (lane >> 2) & 3, tb = lane & 3, h = lane >> 4;
        for (int i = warp; i < n; i += nw) {
            const int la = (int)(signed char)(sp[i * D] >> (8 * ta));
            const int lb = (int)(signed char)(sp[i * D + 1] >> (8 * tb));
            if (la < 0 || lb < 0) continue;
            const int lo = la * LY::stride(0) + lb;
            const float w = sw[(i * D) * KW + ta] * sw[(i * D + 1) * KW + tb];
            for (int c = h; c < cc; c += 2) {
                const float2 uv = su[i * cs + c];
                float* pl = acc + c * 2 * LY::PLANE;
                atomicAdd(pl + lo, w * uv.x);
                atomicAdd(pl + LY::PLANE + lo, w * uv.y);
            }
        }
    } else {
        const int tb = (lane >> 2) & 3, tc = lane & 3, ta0 = lane >> 4;
        for (int i = warp; i < n; i += nw) {
            const int lb = (int)(signed char)(sp[i * D + 1] >> (8 * tb));
            const int lc = (int)(signed char)(sp[i * D + 2] >> (8 * tc));
            if (lb < 0 || lc < 0) continue;
            const float wbc = sw[(i * D + 1) * KW + tb] * sw[(i * D + 2) * KW + tc];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int ta = ta0 + 2 * k;
                const int la = (int)(signed char)(sp[i * D] >> (8 * ta));
                if (la < 0) continue;
                const int lo = la * LY::stride(0) + lb * LY::stride(1 % D) + lc;
                const float w = sw[(i * D) * KW + ta] * wbc;
                for (int c = 0; c < cc; ++c) {
                    const float2 uv = su[i * cs + c];
                    float* pl = acc + c * 2 * LY::PLANE;
                    atomicAdd(pl + lo, w * uv.x);
                    atomicAdd(pl + LY::PLANE + lo, w * uv.y);
                }
            }
        }
    }
    }   // stages
    __syncthreads();
    int P = 1;
#pragma unroll
    for (int d = 0; d < D; ++d) P *= tl.ts[d];
    for (int i = threadIdx.x; i < cc * P; i += blockDim.x) {
        const int c = i / P;
        int r = i - c * P;
        int lidx[MAXD];
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { lidx[d] = r % tl.ts[d]; r /= tl.ts[d]; }
        bool in = true;
        int lo = 0;
        int64_t gflat = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            if (lidx[d] >= e[d]) in = false;
            lo += lidx[d] * LY::stride(d);
            gflat = gflat * geo.g[d] + tunshift(o[d] + lidx[d], tl.sh[d], geo.g[d]);
        }
        if (!in) continue;
        const float* pl = acc + c * 2 * LY::PLANE;
        const float2 v = make_float2(pl[lo], pl[LY::PLANE + lo]);
        float2* dst = grid + (size_t)(c0 + c) * geo.G + gflat;
        if (split) {
            atomicAdd(&dst->x, v.x);
            atomicAdd(&dst->y, v.y);
        } else {
            *dst = v;
        }
    }
}

// Variant in which each warp owns four coils of a single shared accumulator: every warp
// walks all samples of the item for its own coils, so no two warps ever touch the same
// address (no atomics, no private copies), and a sample's geometry is staged once for all
// coils.  Block = 32 * ceil(C / 4) threads.
constexpr int SPW_CW = 4;          // coils per warp

template <int D>
static size_t spread_warpcoil_smem(int C) {
    return (size_t)C * 2 * (D == 2 ? SpL<2>::PLANE : SpL<3>::PLANE) * sizeof(float) +
           (size_t)SP_CHUNK * (C * sizeof(float2) + D * KW * sizeof(float) + D * sizeof(int));
}

template <int D, typename UT>
__global__ void __launch_bounds__(1024)
k_spread_warpcoil(const int* __restrict__ k0t, const float* __restrict__ wt, const UT* __restrict__ u,
                  const int* __restrict__ perm, const int* __restrict__ ext, const int4* __restrict__ items, Geom geo,
                  Tiles tl, float2* __restrict__ grid) {
    using LY = SpL<D>;
    extern __shared__ float smem[];
    const int C = geo.C;
    float* acc = smem;                                              // [C][2][PLANE]
    float2* su = (float2*)(acc + C * 2 * LY::PLANE);                // [SP_CHUNK][C]
    float* sw = (float*)(su + SP_CHUNK * C);                        // [SP_CHUNK][D][KW]
    unsigned* sp = (unsigned*)(sw + SP_CHUNK * D * KW);             // [SP_CHUNK][D]
    const int4 it = items[blockIdx.x];
    const int tile = it.x, beg = it.y, end = it.z;
    const bool split = it.w >= 0;
    int o[MAXD], e[MAXD];
    {
        int r = tile;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            const int tc = r % tl.nt[d];
            r /= tl.nt[d];
            o[d] = tc * tl.ts[d];
            e[d] = min(tl.ts[d], geo.g[d] - o[d]);
        }
    }
    for (int i = threadIdx.x; i < C * 2 * LY::PLANE; i += blockDim.x) acc[i] = 0.f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cw0 = warp * SPW_CW;
    const int ccw = min(SPW_CW, C - cw0);
    for (int sb = beg; sb < end; sb += SP_CHUNK) {   // SP_CHUNK samples at a time
    const int n = min(SP_CHUNK, end - sb);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int s = ext[sb + i];
        const int64_t un = perm ? perm[s] : s;
        for (int c = 0; c < C; ++c) su[i * C + c] = ldc<UT>(u, (size_t)c * geo.M + un);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int p0 = tshift(k0t[(int64_t)d * geo.M + s], tl.sh[d], geo.g[d]);
            unsigned pk = 0;
#pragma unroll
            for (int j = 0; j < KW; ++j) {
                int pp = p0 + j;
                if (pp >= geo.g[d]) pp -= geo.g[d];
                const int l = pp - o[d];
                const unsigned byte = (l >= 0 && l < e[d]) ? (unsigned)l : 0xFFu;
                pk |= byte << (8 * j);
                sw[(i * D + d) * KW + j] = wt[(int64_t)(d * KW + j) * geo.M + s];
            }
            sp[i * D + d] = pk;
        }
    }
    __syncthreads();
    if (D == 2) {
        const int ta = (lane >> 2) & 3, tb = lane & 3, h = lane >> 4;
        const bool has0 = h < ccw, has1 = h + 2 < ccw;
        float* q0 = acc + (cw0 + h) * 2 * LY::PLANE;
        float* q1 = acc + (cw0 + h + 2) * 2 * LY::PLANE;
        for (int i = 0; i < n; ++i) {
            const int la = (int)(signed char)(sp[i * D] >> (8 * ta));
            const int lb = (int)(signed char)(sp[i * D + 1] >> (8 * tb));
            if (la < 0 || lb < 0 || !has0) continue;
            const int lo = la * LY::stride(0) + lb;
            const float w = sw[(i * D) * KW + ta] * sw[(i * D + 1) * KW + tb];
            const float2 u0 = su[i * C + cw0 + h];
            float r0 = q0[lo], i0 = q0[LY::PLANE + lo];
            if (has1) {
                const float2 u1 = su[i * C + cw0 + h + 2];
                float r1 = q1[lo], i1 = q1[LY::PLANE + lo];
                q1[lo] = fmaf(w, u1.x, r1);
                q1[LY::PLANE + lo] = fmaf(w, u1.y, i1);
            }
            q0[lo] = fmaf(w, u0.x, r0);
            q0[LY::PLANE + lo] = fmaf(w, u0.y, i0);
        }
    } else {
        const int tb = (lane >> 2) & 3, tc = lane & 3, ta0 = lane >> 4;
        for (int i = 0; i < n; ++i) {
            const int lb = (int)(signed char)(sp[i * D + 1] >> (8 * tb));
            const int lc = (int)(signed char)(sp[i * D + 2] >> (8 * tc));
            if (lb < 0 || lc < 0) continue;
            const float wbc = sw[(i * D + 1) * KW + tb] * sw[(i * D + 2) * KW + tc];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int ta = ta0 + 2 * k;
                const int la = (int)(signed char)(sp[i * D] >> (8 * ta));
                if (la < 0) continue;
                const int lo = la * LY::stride(0) + lb * LY::stride(1 % D) + lc;
                const float w = sw[(i * D) * KW + ta] * wbc;
                float rr[SPW_CW], ii[SPW_CW];
#pragma unroll
                for (int c = 0; c < SPW_CW; ++c)
                    if (c < ccw) { float* pl = acc + (cw0 + c) * 2 * LY::PLANE; rr[c] = pl[lo]; ii[c] = pl[LY::PLANE + lo]; }
#pragma unroll
                for (int c = 0; c < SPW_CW; ++c)
                    if (c < ccw) {
                        const float2 uv = su[i * C + cw0 + c];
                        float* pl = acc + (cw0 + c) * 2 * LY::PLANE;
                        pl[lo] = fmaf(w, uv.x, rr[c]);
                        pl[LY::PLANE + lo] = fmaf(w, uv.y, ii[c]);
                    }
            }
        }
    }
    }   // stages
    __syncthreads();
    int P = 1;
#pragma unroll
    for (int d = 0; d < D; ++d) P *= tl.ts[d];
    for (int i = threadIdx.x; i < C * P; i += blockDim.x) {
        const int c = i / P;
        int r = i - c * P;
        int lidx[MAXD];
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { lidx[d] = r % tl.ts[d]; r /= tl.ts[d]; }
        bool in = true;
        int lo = 0;
        int64_t gflat = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            if (lidx[d] >= e[d]) in = false;
            lo += lidx[d] * LY::stride(d);
            gflat = gflat * geo.g[d] + tunshift(o[d] + lidx[d], tl.sh[d], geo.g[d]);
        }
        if (!in) continue;
        const float* pl = acc + c * 2 * LY::PLANE;
        const float2 v = make_float2(pl[lo], pl[LY::PLANE + lo]);
        float2* dst = grid + (size_t)c * geo.G + gflat;
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
__device__ __forceinline__ void zero_split_body(const int* __restrict__ split_tiles, const Geom& geo, const Tiles& tl,
                                                int P, float2* __restrict__ grid, int b) {
    const int tile = split_tiles[b];
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

template <int D>
__global__ void k_zero_split(const int* __restrict__ split_tiles, Geom geo, Tiles tl, int P, float2* __restrict__ grid) {
    zero_split_body<D>(split_tiles, geo, tl, P, grid, blockIdx.x);
}

// ---------------------------------------------------------------- adjoint: post
template <int D, typename MT>
__global__ void k_adj_image(const float2* __restrict__ grid, const MT* __restrict__ maps, const float* __restrict__ apod,
                            Geom geo, float2* __restrict__ x) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= geo.N) return;
    x[j] = adj_pixel<D, MT>(grid, maps, apod, geo, j);
}

// Image coordinates of pixel j and the strides of its axes (slowest axis first).
template <int D>
__device__ __forceinline__ void pix_coords(int64_t j, const Geom& geo, int* jj, int64_t* stride) {
    int64_t r = j, s = 1;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) {
        jj[d] = (int)(r % geo.n[d]);
        r /= geo.n[d];
        stride[d] = s;
        s *= geo.n[d];
    }
}

// TV dual step (Sec. 4.2): v_k[j] <- projection of v_k[j] + sigma (xbar[j + e_k] - xbar[j])
// onto |v| <= lambda (periodic forward differences).  Each thread owns v at its pixel and only
// reads xbar, so the update is in place.
template <int D>
__global__ void k_tv_dual(const float2* __restrict__ xbar, float2* __restrict__ v, Geom geo,
                          const float* __restrict__ sched, const int* __restrict__ iter, float lambda) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= geo.N) return;
    const float sigma = sched[3 * (*iter)];
    int jj[D];
    int64_t stride[D];
    pix_coords<D>(j, geo, jj, stride);
    const float2 xc = xbar[j];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const int64_t jn = jj[k] + 1 < geo.n[k] ? j + stride[k] : j - (int64_t)(geo.n[k] - 1) * stride[k];
        const float2 xn = xbar[jn];
        float2 z = v[(size_t)k * geo.N + j];
        z.x += sigma * (xn.x - xc.x);
        z.y += sigma * (xn.y - xc.y);
        const float m = sqrtf(z.x * z.x + z.y * z.y);
        if (m > lambda) {
            const float sc = lambda / m;
            z.x *= sc;
            z.y *= sc;
        }
        v[(size_t)k * geo.N + j] = z;
    }
}

// Primal step: z = x - tau A^H u; l2 prox z/(1 + tau lambda) and extrapolation fused
// (REG == 0, Sec. 4.1); for the wavelet prox (REG == 1) z is written for the DWT; for TV
// (REG == 2, Sec. 4.2) x <- z - tau G^H v, G^H v = sum_k (v_k[j - e_k] - v_k[j]), and the
// extrapolation.
template <int D, typename MT, int REG>
__device__ __forceinline__ void adj_primal_body(const float2* __restrict__ grid, const MT* __restrict__ maps,
                                                const float* __restrict__ apod, const Geom& geo,
                                                float2* __restrict__ x, float2* __restrict__ xbar,
                                                float2* __restrict__ z, const float* __restrict__ sched,
                                                const int* __restrict__ iter, float lambda,
                                                const float2* __restrict__ v, int64_t j) {
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
    } else if (REG == 2) {
        int jj[D];
        int64_t stride[D];
        pix_coords<D>(j, geo, jj, stride);
        float2 gh = make_float2(0.f, 0.f);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int64_t jm = jj[a] > 0 ? j - stride[a] : j + (int64_t)(geo.n[a] - 1) * stride[a];
            const float2 vm = v[(size_t)a * geo.N + jm], vc = v[(size_t)a * geo.N + j];
            gh.x += vm.x - vc.x;
            gh.y += vm.y - vc.y;
        }
        const float2 xn = make_float2(zz.x - tau * gh.x, zz.y - tau * gh.y);
        xbar[j] = make_float2(xn.x + theta * (xn.x - xo.x), xn.y + theta * (xn.y - xo.y));
        x[j] = xn;
    } else {
        z[j] = zz;
    }
}

template <int D, typename MT, int REG>
__global__ void k_adj_primal(const float2* __restrict__ grid, const MT* __restrict__ maps, const float* __restrict__ apod,
                             Geom geo, float2* __restrict__ x, float2* __restrict__ xbar, float2* __restrict__ z,
                             const float* __restrict__ sched, const int* __restrict__ iter, float lambda,
                             const float2* __restrict__ v) {
    adj_primal_body<D, MT, REG>(grid, maps, apod, geo, x, xbar, z, sched, iter, lambda, v,
                                (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
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

// The grid FFTs of the NUFFT pair: the own 3D passes when the plan has them, else cuFFT.
static kp_status grid_fft_forward(kp_plan p, cudaStream_t st) {
    if (p->fft3) return fft3_forward(p, p->d_grid, p->d_gridF, st);
    KP_TRY_CUFFT(cufftSetStream(p->fft, st));
    KP_TRY_CUFFT(cufftExecC2C(p->fft, (cufftComplex*)p->d_grid, (cufftComplex*)p->d_gridF, CUFFT_FORWARD));
    return KP_OK;
}

static kp_status grid_fft_inverse(kp_plan p, cudaStream_t st) {
    if (p->fft3) return fft3_inverse(p, p->d_grid2, st);
    KP_TRY_CUFFT(cufftSetStream(p->fft, st));
    KP_TRY_CUFFT(cufftExecC2C(p->fft, (cufftComplex*)p->d_grid2, (cufftComplex*)p->d_grid2, CUFFT_INVERSE));
    return KP_OK;
}

kp_status fill_image(float2* x, int64_t n, float2 v, cudaStream_t st) {
    k_fill<<<nblk(n, 256), 256, 0, st>>>(x, n, v);
    KP_LAUNCH_CHECK();
    return KP_OK;
}

static kp_status fwd_grid(kp_plan p, const float2* x, cudaStream_t st) {
    const Geom& g = p->geo;
    if (p->fft3) {                      // the own FFT's first pass forms the pre-step itself
        mark(p, PH_FFT_FWD, st);
        return fft3_forward_image(p, x, st);
    }
    const kp_cdtype mt = p->unit_maps ? KP_C64 : p->maps_t;
    mark(p, PH_FWD_PRE, st);
    p->launches += 1;
    KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(mt, MT,
        k_fwd_pre<DD, MT><<<nblk(g.G, 256), 256, 0, st>>>(x, p->unit_maps ? nullptr : (const MT*)p->d_maps,
                                                         p->d_apod, g, p->d_grid)));
    KP_LAUNCH_CHECK();
    mark(p, PH_FFT_FWD, st);
    return grid_fft_forward(p, st);
}

// Forward grid spectrum of x (pre-step into d_grid, FFT into d_gridF), no interpolation.
kp_status forward_grid_only(kp_plan p, const float2* x, cudaStream_t st) { return fwd_grid(p, x, st); }

// Forward pre-step only (coil multiply, apodise, pad) of x into d_grid.
kp_status pre_only(kp_plan p, const float2* x, cudaStream_t st) {
    const Geom& g = p->geo;
    if (p->fft3) return KP_OK;          // the own FFT forms the pre-step from the image itself
    const kp_cdtype mt = p->unit_maps ? KP_C64 : p->maps_t;
    p->launches += 1;
    KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(mt, MT,
        k_fwd_pre<DD, MT><<<nblk(g.G, 256), 256, 0, st>>>(x, p->unit_maps ? nullptr : (const MT*)p->d_maps,
                                                         p->d_apod, g, p->d_grid)));
    KP_LAUNCH_CHECK();
    return KP_OK;
}

// Forward FFT of a grid already written into d_grid (the fused primal kernel writes the next
// iteration's pre-step there).
kp_status fft_forward_only(kp_plan p, cudaStream_t st) {
    mark(p, PH_FFT_FWD, st);
    if (p->fft3) return fft3_forward_image(p, p->d_xbar, st);   // the pre-step of xbar, fused
    return grid_fft_forward(p, st);
}

kp_status fft_inverse_only(kp_plan p, cudaStream_t st) {
    mark(p, PH_FFT_INV, st);
    return grid_fft_inverse(p, st);
}

template <int MODE>
static kp_status launch_interp(kp_plan p, kp_cdtype t, const InterpIO& io, cudaStream_t st) {
    const Geom& g = p->geo;
    const size_t rt = g.D == 2 ? IpL<2>::PER_COIL : IpL<3>::PER_COIL;
    const size_t smem = (size_t)IP_CH * rt * sizeof(float2);
    const dim3 grid((unsigned)p->n_iitems, (g.C + IP_CH - 1) / IP_CH);
    static PerDeviceOnce attr[2][3][3];
    mark(p, PH_INTERP, st);
    p->launches += 1;
    if (p->n_iitems == 0) return KP_OK;
    if (p->chunk > IP_THREADS) { set_error("interpolation items larger than the block"); return KP_EINTERNAL; }
    KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(t, T,
        if (attr[DD - 2][MODE][t].first())
            KP_TRY_CUDA(cudaFuncSetAttribute(k_interp_tile<DD, MODE, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
        k_interp_tile<DD, MODE, T><<<grid, IP_THREADS, smem, st>>>(p->d_iitems, p->d_k0, p->d_wt, p->d_gridF, g, p->tiles, io)));
    KP_LAUNCH_CHECK();
    return KP_OK;
}

kp_status forward_to(kp_plan p, const float2* x, void* out, kp_cdtype out_t, const int* perm, cudaStream_t st) {
    KP_TRY(fwd_grid(p, x, st));
    InterpIO io{};
    io.out = out;
    io.perm = perm;
    io.flag = p->d_flag + KP_FLAG_TIMEOUT;
    io.wait = p->wait_cycles;
    return launch_interp<0>(p, out_t, io, st);
}

kp_status forward_scaled(kp_plan p, const float2* x, float2* out_sorted, const float* ps, cudaStream_t st,
                         const double* n2) {
    KP_TRY(fwd_grid(p, x, st));
    InterpIO io{};
    io.outs = out_sorted;
    io.ps = ps;
    io.n2 = n2;
    io.flag = p->d_flag + KP_FLAG_TIMEOUT;
    io.wait = p->wait_cycles;
    return launch_interp<1>(p, KP_C64, io, st);
}

kp_status forward_dual(kp_plan p, const float2* xbar, cudaStream_t st) {
    KP_TRY(fwd_grid(p, xbar, st));
    return interp_dual_only(p, st);
}

kp_status interp_dual_only(kp_plan p, cudaStream_t st) {
    InterpIO io{};
    io.ys = p->d_ys;
    io.flag = p->d_flag + KP_FLAG_TIMEOUT;
    io.wait = p->wait_cycles;
    io.ps = p->d_ps;
    io.u = p->d_u;
    io.sched = p->d_sched;
    io.iter = p->d_iter;
    return launch_interp<2>(p, p->ys_t, io, st);
}

// Interleaved-pair spreading with NW warps (variants 6, 7).
template <int D, typename UT, int NW>
static kp_status launch_spread_v(kp_plan p, const UT* u, const int* perm, cudaStream_t st) {
    static PerDeviceOnce attr;
    const size_t sm = spread_v_smem<D, NW>();
    if (attr.first()) KP_TRY_CUDA(cudaFuncSetAttribute(k_spread_v<D, UT, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const Geom& g = p->geo;
    k_spread_v<D, UT, NW><<<dim3((unsigned)p->n_items, (g.C + 3) / 4), NW * 32, sm, st>>>(
        p->d_k0, p->d_wt, u, perm, p->d_ext, p->d_items, g, p->tiles, p->d_grid2);
    return KP_OK;
}

// Two-phase spreading, 3D only (variants 10, 11): padded tiles into the slots, then gather.
// Two-phase spreading, 2D (variant 12): padded tiles of 4 coils into the slots, then gather.
template <typename UT>
static kp_status launch_spread_own2(kp_plan p, const UT* u, const int* perm, cudaStream_t st) {
    const Geom& g = p->geo;
    if (g.D != 2 || !p->d_halo || p->halo_cap < (size_t)p->n_oitems * g.C * PT2SQ) {
        set_error("two-phase spreading needs a 2D plan with its slot storage");
        return KP_EINTERNAL;
    }
    static PerDeviceOnce attr;
    const size_t sm = spread_own2_smem<4>();
    if (attr.first())
        KP_TRY_CUDA(cudaFuncSetAttribute(k_spread_own2<UT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    if (p->n_oitems > 0)
        k_spread_own2<UT, 4><<<dim3((unsigned)p->n_oitems, (g.C + 3) / 4), 128, sm, st>>>(
            p->d_k0, p->d_wt, u, perm, p->d_oitems, g, p->tiles, p->d_halo);
    KP_LAUNCH_CHECK();
    mark(p, PH_SPREAD_RED, st);
    const dim3 gg((unsigned)(((g.g[1] + 255) / 256) * g.g[0]), (unsigned)g.C);
    k_halo_gather2<<<gg, 256, 0, st>>>(p->d_halo, p->d_tslot, g, p->tiles, p->d_grid2);
    p->launches += 1;
    return KP_OK;
}

template <int D, typename UT, int NP>
static kp_status launch_spread_own(kp_plan p, const UT* u, const int* perm, cudaStream_t st) {
    const Geom& g = p->geo;
    if (D != 3 || !p->d_halo || p->halo_cap < (size_t)p->n_oitems * g.C * SL_P || p->tiles.ts[0] > 8 ||
        p->tiles.ts[1] > 8 || p->tiles.ts[2] > 8) {
        set_error("two-phase spreading needs a 3D plan with tiles of at most 8 and its slot storage");
        return KP_EINTERNAL;
    }
    static PerDeviceOnce attr;
    const size_t sm = spread_own_smem<NP>();
    if (attr.first()) KP_TRY_CUDA(cudaFuncSetAttribute(k_spread_own<UT, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    if (p->n_oitems > 0)
        k_spread_own<UT, NP><<<dim3((unsigned)p->n_oitems, (g.C + 2 * NP - 1) / (2 * NP)), NP * 64, sm, st>>>(
            p->d_k0, p->d_wt, u, perm, p->d_oitems, g, p->tiles, p->d_halo);
    KP_LAUNCH_CHECK();
    mark(p, PH_SPREAD_RED, st);
    k_halo_gather<<<(unsigned)p->tiles.ntiles, 256, 0, st>>>(p->d_halo, p->d_tslot, g, p->tiles, p->d_grid2);
    KP_LAUNCH_CHECK();
    p->launches += 1;
    return KP_OK;
}

// Allocates the slot storage of the two-phase variants if it fits a budget (a quarter of
// the free device memory, at most 16 GiB); false when it does not.
static bool ensure_halo(kp_plan p) {
    const Geom& g = p->geo;
    if (p->n_oitems == 0) return false;
    const size_t need = (size_t)p->n_oitems * g.C * (g.D == 3 ? SL_P : PT2SQ);
    if (p->d_halo && p->halo_cap >= need) return true;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return false;
    if (need * sizeof(float2) > std::min(fr / 4, (size_t)16 << 30)) return false;
    if (p->d_halo) cudaFree(p->d_halo);
    p->d_halo = nullptr;
    p->halo_cap = 0;
    if (cudaMalloc(&p->d_halo, need * sizeof(float2)) != cudaSuccess) { cudaGetLastError(); p->d_halo = nullptr; return false; }
    p->halo_cap = need;
    return true;
}

// Plane-owner spreading, 3D only (variants 8, 9).
template <int D, typename UT, int CG>
static kp_status launch_spread_z(kp_plan p, const UT* u, const int* perm, cudaStream_t st) {
    if (D != 3) { set_error("spreading variants 8 and 9 are 3D only"); return KP_EINTERNAL; }
    static PerDeviceOnce attr;
    const size_t sm = spread_z_smem<CG>();
    if (attr.first()) KP_TRY_CUDA(cudaFuncSetAttribute(k_spread_z<UT, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const Geom& g = p->geo;
    k_spread_z<UT, CG><<<dim3((unsigned)p->n_items, (g.C + CG - 1) / CG), 256, sm, st>>>(
        p->d_k0, p->d_wt, u, perm, p->d_ext, p->d_items, g, p->tiles, p->d_grid2);
    return KP_OK;
}

// Private-copy spreading with CH coils per CTA and NW warps (variants 0, 3, 4, 5).
template <int D, typename UT, int CH, int NW>
static kp_status launch_spread_priv(kp_plan p, const UT* u, const int* perm, cudaStream_t st) {
    static PerDeviceOnce attr;
    const size_t sm = spread_smem<D, CH, NW>();
    if (attr.first()) KP_TRY_CUDA(cudaFuncSetAttribute(k_spread<D, UT, CH, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const Geom& g = p->geo;
    k_spread<D, UT, CH, NW><<<dim3((unsigned)p->n_items, (g.C + CH - 1) / CH), NW * 32, sm, st>>>(
        p->d_k0, p->d_wt, u, perm, p->d_ext, p->d_items, g, p->tiles, p->d_grid2);
    return KP_OK;
}

kp_status zero_split_only(kp_plan p, cudaStream_t st) {
    const Geom& g = p->geo;
    int P = 1;
    for (int d = 0; d < g.D; ++d) P *= p->tiles.ts[d];
    if (p->spread_tuned && p->spread_variant >= 10) return KP_OK;   // two-phase spreading stores every point
    if (p->n_split > 0) {
        KP_DISPATCH_D(g.D, DD, k_zero_split<DD><<<(unsigned)p->n_split, 256, 0, st>>>(p->d_split, g, p->tiles, P,
                                                                                      p->d_grid2));
        KP_LAUNCH_CHECK();
        p->launches += 1;
    }
    return KP_OK;
}

// The spreading kernels alone (no inverse FFT).
static kp_status spread_only(kp_plan p, const void* u, kp_cdtype u_t, const int* perm, cudaStream_t st,
                             bool splits_zeroed) {
    const Geom& g = p->geo;
    mark(p, PH_SPREAD, st);
    if (!splits_zeroed && p->spread_variant < 10) KP_TRY(zero_split_only(p, st));   // 10, 11 store every point
    p->launches += 1;
    if (p->spread_variant == 0 || p->spread_variant >= 3) {
        KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(u_t, UT,
            switch (p->spread_variant) {
                case 0: KP_TRY((launch_spread_priv<DD, UT, 4, 4>(p, (const UT*)u, perm, st))); break;
                case 3: KP_TRY((launch_spread_priv<DD, UT, 2, 8>(p, (const UT*)u, perm, st))); break;
                case 4: KP_TRY((launch_spread_priv<DD, UT, 1, 8>(p, (const UT*)u, perm, st))); break;
                case 6: KP_TRY((launch_spread_v<DD, UT, 4>(p, (const UT*)u, perm, st))); break;
                case 7: KP_TRY((launch_spread_v<DD, UT, 8>(p, (const UT*)u, perm, st))); break;
                case 8: KP_TRY((launch_spread_z<DD, UT, 8>(p, (const UT*)u, perm, st))); break;
                case 9: KP_TRY((launch_spread_z<DD, UT, 4>(p, (const UT*)u, perm, st))); break;
                case 10: KP_TRY((launch_spread_own<DD, UT, 4>(p, (const UT*)u, perm, st))); break;
                case 11: KP_TRY((launch_spread_own<DD, UT, 2>(p, (const UT*)u, perm, st))); break;
                case 12: KP_TRY((launch_spread_own2<UT>(p, (const UT*)u, perm, st))); break;
                default: KP_TRY((launch_spread_priv<DD, UT, 2, 4>(p, (const UT*)u, perm, st))); break;
            }));
    } else if (p->spread_variant == 2) {
        static PerDeviceOnce attr_w[2][3];
        const size_t sm = g.D == 2 ? spread_warpcoil_smem<2>(g.C) : spread_warpcoil_smem<3>(g.C);
        const unsigned nthr = 32u * (unsigned)((g.C + SPW_CW - 1) / SPW_CW);
        KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(u_t, UT,
            if (attr_w[DD - 2][u_t].first())
                KP_TRY_CUDA(cudaFuncSetAttribute(k_spread_warpcoil<DD, UT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
            k_spread_warpcoil<DD, UT><<<(unsigned)p->n_items, nthr, sm, st>>>(
                p->d_k0, p->d_wt, (const UT*)u, perm, p->d_ext, p->d_items, g, p->tiles, p->d_grid2)));
    } else {
        static PerDeviceOnce attr_a[2][3];
        KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(u_t, UT,
            if (attr_a[DD - 2][u_t].first())
                KP_TRY_CUDA(cudaFuncSetAttribute(k_spread_atomic<DD, UT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
            k_spread_atomic<DD, UT><<<dim3((unsigned)p->n_items, (g.C + SPA_CH - 1) / SPA_CH), SPA_THREADS,
                                      spread_atomic_smem<DD>(std::min(g.C, SPA_CH)), st>>>(
                p->d_k0, p->d_wt, (const UT*)u, perm, p->d_ext, p->d_items, g, p->tiles, p->d_grid2)));
    }
    KP_LAUNCH_CHECK();
    return KP_OK;
}

kp_status adjoint_to_grid(kp_plan p, const void* u, kp_cdtype u_t, const int* perm, cudaStream_t st,
                          bool splits_zeroed) {
    KP_TRY(spread_only(p, u, u_t, perm, st, splits_zeroed));
    mark(p, PH_FFT_INV, st);
    return grid_fft_inverse(p, st);
}

// Picks the spreading variant and the samples per work item by timing the spreading kernels
// on the plan's own work items (values do not affect the cost; once per plan, at its first
// trajectory).  Variants: 0 private copies, 4 coils x 4 warps; 1 shared atomics; 2 warp per
// 4 coils; 3 private, 2 coils x 8 warps; 4 private, 1 coil x 8 warps; 5 private, 2 coils x 4
// warps; 6, 7 private interleaved coil pairs, 4 coils x 4 / 8 warps; 8, 9 (3D) z-plane owners,
// 8 / 4 coils; 10, 11 (3D) two-phase padded tiles + gather, 8 / 4 coils, and 12 (2D) two-phase
// with warp-private padded tiles (when their slot storage fits).  Larger items mean fewer split tiles (fewer global atomics) but fewer, longer CTAs.
kp_status autotune_spread(kp_plan p, cudaStream_t st) {
    if (p->spread_tuned) {
        // a new trajectory may need more slots than the two-phase variants hold: fall back to the
        // private-copy variant, whose lists were not built for a two-phase plan
        if (p->spread_variant >= 10 && !ensure_halo(p)) {
            p->spread_variant = 0;
            KP_TRY(build_spread_lists(p, st));
        }
        return KP_OK;
    }
    int force_v = -1, force_c = 0;
    if (const char* ev = getenv("KPDHG_SPREAD_VARIANT")) force_v = atoi(ev);   // tuning overrides
    if (const char* ev = getenv("KPDHG_SPREAD_CHUNK")) force_c = atoi(ev);
    const Geom& g = p->geo;
    const bool wc_ok = (g.D == 2 ? spread_warpcoil_smem<2>(g.C) : spread_warpcoil_smem<3>(g.C)) <= 220 * 1024;
    const bool own_ok = ensure_halo(p);
    const auto applies = [&](int v) {
        if (v == 2) return wc_ok;
        if (v >= 8 && v <= 11) return g.D == 3 && (v < 10 || own_ok);
        if (v == 12) return g.D == 2 && own_ok;
        return v >= 0 && v <= 7;
    };
    if (!applies(force_v)) force_v = -1;
    if (force_c < SP_CHUNK || force_c % SP_CHUNK != 0) force_c = 0;
    std::vector<int> chunks;
    if (force_c) chunks.push_back(force_c);
    else chunks = {256, 1024, 4096};
    std::vector<int> variants;
    if (force_v >= 0) variants.push_back(force_v);
    else for (int v = 0; v <= 12; ++v) if (applies(v)) variants.push_back(v);
    if (chunks.size() == 1 && variants.size() == 1) {
        p->spread_variant = variants[0];
        if (chunks[0] != p->spread_chunk) KP_TRY(build_spread_items(p, chunks[0], st));
        p->spread_tuned = true;
        return KP_OK;
    }
    KP_TRY_CUDA(cudaMemsetAsync(p->d_kt, 0, (size_t)g.C * g.M * sizeof(float2), st));
    cudaEvent_t e0, e1;
    KP_TRY_CUDA(cudaEventCreate(&e0));
    KP_TRY_CUDA(cudaEventCreate(&e1));
    // The spreading kernels alone are timed (the inverse FFT is the same for every choice),
    // in two interleaved rounds, keeping each configuration's faster round: one round alone
    // was noisy enough to pick a variant 20 % slower than the best.
    std::vector<float> t_min(chunks.size() * variants.size(), 1e30f);
    const bool prof = p->profiling;
    p->profiling = false;
    kp_status status = KP_OK;
    for (int round = 0; round < 2 && status == KP_OK; ++round) {
        for (size_t ci = 0; ci < chunks.size() && status == KP_OK; ++ci) {
            const int c = chunks[ci];
            if (c != p->spread_chunk) status = build_spread_items(p, c, st);
            for (size_t vi = 0; vi < variants.size() && status == KP_OK; ++vi) {
                const int v = variants[vi];
                if (v >= 10 && ci != 0) continue;   // the two-phase variants ignore the item size
                p->spread_variant = v;
                status = spread_only(p, p->d_kt, KP_C64, nullptr, st, true);
                if (status != KP_OK) break;
                cudaEventRecord(e0, st);
                for (int r = 0; r < 4 && status == KP_OK; ++r) status = spread_only(p, p->d_kt, KP_C64, nullptr, st, true);
                cudaEventRecord(e1, st);
                if (status != KP_OK || cudaEventSynchronize(e1) != cudaSuccess) { status = status != KP_OK ? status : KP_ECUDA; break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                float& tm = t_min[ci * variants.size() + vi];
                tm = std::min(tm, ms);
            }
        }
    }
    float best = 1e30f;
    int best_v = 0, best_c = p->spread_chunk;
    for (size_t ci = 0; ci < chunks.size(); ++ci)
        for (size_t vi = 0; vi < variants.size(); ++vi)
            if (t_min[ci * variants.size() + vi] < best) {
                best = t_min[ci * variants.size() + vi];
                best_v = variants[vi];
                best_c = chunks[ci];
            }
    p->profiling = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    KP_TRY(status);
    p->spread_variant = best_v;
    if (best_c != p->spread_chunk) KP_TRY(build_spread_items(p, best_c, st));
    p->spread_tuned = true;
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
                                                                   p->d_xbar, p->d_z, p->d_sched, p->d_iter, lambda,
                                                                   nullptr)));
    } else if (reg == KP_REG_TV) {
        // dual step on v from the current xbar, then the primal step reading the new v
        if (!p->d_v) { set_error("TV dual variable not allocated"); return KP_EINTERNAL; }
        p->launches += 1;
        KP_DISPATCH_D(g.D, DD,
            k_tv_dual<DD><<<nblk(g.N, 256), 256, 0, st>>>(p->d_xbar, p->d_v, g, p->d_sched, p->d_iter, lambda));
        KP_LAUNCH_CHECK();
        KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(mt, MT,
            k_adj_primal<DD, MT, 2><<<nblk(g.N, 256), 256, 0, st>>>(p->d_grid2, (const MT*)p->d_maps, p->d_apod, g, p->d_x,
                                                                   p->d_xbar, p->d_z, p->d_sched, p->d_iter, lambda,
                                                                   p->d_v)));
    } else {
        KP_DISPATCH_D(g.D, DD, KP_DISPATCH_T(mt, MT,
            k_adj_primal<DD, MT, 1><<<nblk(g.N, 256), 256, 0, st>>>(p->d_grid2, (const MT*)p->d_maps, p->d_apod, g, p->d_x,
                                                                   p->d_xbar, p->d_z, p->d_sched, p->d_iter, lambda,
                                                                   nullptr)));
    }
    KP_LAUNCH_CHECK();
    return KP_OK;
}

// sum_k sum_j |x[j + e_k] - x[j]| (float64) added into *out.
template <int D>
__global__ void k_tv_sumabs(const float2* __restrict__ x, Geom geo, double* __restrict__ out) {
    __shared__ double ws[32];
    double s = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < geo.N; j += (int64_t)gridDim.x * blockDim.x) {
        int jj[D];
        int64_t stride[D];
        pix_coords<D>(j, geo, jj, stride);
        const float2 xc = x[j];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int64_t jn = jj[k] + 1 < geo.n[k] ? j + stride[k] : j - (int64_t)(geo.n[k] - 1) * stride[k];
            const float2 xn = x[jn];
            const double dx = (double)xn.x - xc.x, dy = (double)xn.y - xc.y;
            s += sqrt(dx * dx + dy * dy);
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = s;
    __syncthreads();
    if (w == 0) {
        s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) atomicAdd(out, s);
    }
}

kp_status tv_sumabs(kp_plan p, const float2* x, double* out, cudaStream_t st) {
    const Geom& g = p->geo;
    const unsigned b = (unsigned)std::min<int64_t>(nblk(g.N, 256), 1216);
    p->launches += 1;
    KP_DISPATCH_D(g.D, DD, k_tv_sumabs<DD><<<b, 256, 0, st>>>(x, g, out));
    KP_LAUNCH_CHECK();
    return KP_OK;
}

// ---------------------------------------------------------------- batched phases
template <int D>
__global__ void k_zero_split_b(const BZero* __restrict__ cs, const int* __restrict__ boff, int ncase) {
    const int c = batch_case(boff, ncase, (int)blockIdx.x);
    const BZero& a = cs[c];
    zero_split_body<D>(a.split, a.geo, a.tl, a.P, a.grid, (int)blockIdx.x - boff[c]);
}

template <int D, typename MT>
__global__ void k_adj_primal_b(const BPrimal* __restrict__ cs, const int* __restrict__ boff, int ncase) {
    const int c = batch_case(boff, ncase, (int)blockIdx.x);
    const BPrimal& a = cs[c];
    const int64_t j = (int64_t)((int)blockIdx.x - boff[c]) * blockDim.x + threadIdx.x;
    if (a.reg == 0)
        adj_primal_body<D, MT, 0>(a.grid, (const MT*)a.maps, a.apod, a.geo, a.x, a.xbar, a.z, a.sched, a.iter, a.lambda,
                                  nullptr, j);
    else
        adj_primal_body<D, MT, 1>(a.grid, (const MT*)a.maps, a.apod, a.geo, a.x, a.xbar, a.z, a.sched, a.iter, a.lambda,
                                  nullptr, j);
}

template <int D, typename MT>
__global__ void k_fwd_pre_b(const BPre* __restrict__ cs, const int* __restrict__ boff, int ncase) {
    const int c = batch_case(boff, ncase, (int)blockIdx.x);
    const BPre& a = cs[c];
    fwd_pre_body<D, MT>(a.x, (const MT*)a.maps, a.apod, a.geo, a.grid,
                        (int64_t)((int)blockIdx.x - boff[c]) * blockDim.x + threadIdx.x);
}

// Every case's iteration counter += 1 (descriptor = the counter's address).
__global__ void k_advance_b(int* const* __restrict__ iters, int ncase) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncase) *iters[c] += 1;
}

kp_status phase_upload(BatchPhase& ph, const void* descs, size_t desc_bytes, int ncase, const std::vector<int>& boff) {
    if (desc_bytes > ph.desc_cap) {
        if (ph.d_desc) cudaFree(ph.d_desc);
        ph.d_desc = nullptr;
        ph.desc_cap = 0;
        KP_TRY_CUDA(cudaMalloc(&ph.d_desc, desc_bytes));
        ph.desc_cap = desc_bytes;
    }
    if (boff.size() > ph.boff_cap) {
        if (ph.d_boff) cudaFree(ph.d_boff);
        ph.d_boff = nullptr;
        ph.boff_cap = 0;
        KP_TRY_CUDA(cudaMalloc(&ph.d_boff, boff.size() * sizeof(int)));
        ph.boff_cap = boff.size();
    }
    if (desc_bytes) KP_TRY_CUDA(cudaMemcpy(ph.d_desc, descs, desc_bytes, cudaMemcpyHostToDevice));
    if (!boff.empty()) KP_TRY_CUDA(cudaMemcpy(ph.d_boff, boff.data(), boff.size() * sizeof(int), cudaMemcpyHostToDevice));
    ph.ncase = ncase;
    ph.nblocks = boff.empty() ? 0u : (unsigned)boff.back();
    return KP_OK;
}

void phase_free(BatchPhase& ph) {
    if (ph.d_desc) cudaFree(ph.d_desc);
    if (ph.d_boff) cudaFree(ph.d_boff);
    ph = BatchPhase{};
}

void batch_iter_free(BatchIter& bi) {
    for (BatchPhase* ph : {&bi.interp, &bi.zero, &bi.spread, &bi.primal, &bi.pre, &bi.advance}) phase_free(*ph);
    for (auto& ph : bi.fwd) phase_free(ph);
    for (auto& ph : bi.inv) phase_free(ph);
    bi.fwd.clear();
    bi.inv.clear();
    bi.built = false;
}

// Descriptors of `sel` cases with `blocks(case)` blocks each, uploaded into ph.
template <typename DESC, typename MAKE, typename BLOCKS>
static kp_status build_phase(const std::vector<kp_plan>& ps, const std::vector<int>& sel, BatchPhase& ph, MAKE make,
                             BLOCKS blocks) {
    std::vector<DESC> ds;
    std::vector<int> boff(1, 0);
    for (int i : sel) {
        const int64_t nb = blocks(ps[i]);
        if (nb <= 0) continue;
        if ((int64_t)boff.back() + nb > INT32_MAX) { set_error("batched launch larger than 2^31 blocks"); return KP_EINVAL; }
        ds.push_back(make(ps[i], i));
        boff.push_back(boff.back() + (int)nb);
    }
    return phase_upload(ph, ds.data(), ds.size() * sizeof(DESC), (int)ds.size(), boff);
}

kp_status batch_nufft_build(const std::vector<kp_plan>& ps, const std::vector<int>& regs, const std::vector<float>& lams,
                            BatchIter& bi) {
    const int n = (int)ps.size();
    std::vector<int> all(n), l2;
    for (int i = 0; i < n; ++i) {
        all[i] = i;
        if (regs[i] == KP_REG_L2) l2.push_back(i);
    }
    bi.yt = ps[0]->ys_t;
    bi.mt = ps[0]->maps_t;
    auto cgroups = [](kp_plan p, int per) { return (int64_t)((p->geo.C + per - 1) / per); };
    KP_TRY(build_phase<BInterp>(ps, all, bi.interp, [&](kp_plan p, int) {
        BInterp a{};
        a.items = p->d_iitems;
        a.k0t = p->d_k0;
        a.wt = p->d_wt;
        a.grid = p->d_gridF;
        a.geo = p->geo;
        a.tl = p->tiles;
        a.io.ys = p->d_ys;
        a.io.flag = p->d_flag + KP_FLAG_TIMEOUT;
        a.io.wait = p->wait_cycles;
        a.io.ps = p->d_ps;
        a.io.u = p->d_u;
        a.io.sched = p->d_sched;
        a.io.iter = p->d_iter;
        a.nx = (int)p->n_iitems;
        return a;
    }, [&](kp_plan p) { return p->n_iitems * cgroups(p, IP_CH); }));
    KP_TRY(build_phase<BZero>(ps, all, bi.zero, [&](kp_plan p, int) {
        BZero a{};
        a.split = p->d_split;
        a.geo = p->geo;
        a.tl = p->tiles;
        a.P = 1;
        for (int d = 0; d < p->geo.D; ++d) a.P *= p->tiles.ts[d];
        a.grid = p->d_grid2;
        return a;
    }, [&](kp_plan p) { return p->n_split; }));
    KP_TRY(build_phase<BSpread>(ps, all, bi.spread, [&](kp_plan p, int) {
        BSpread a{};
        a.k0t = p->d_k0;
        a.wt = p->d_wt;
        a.u = p->d_u;
        a.perm = nullptr;
        a.ext = p->d_ext;
        a.items = p->d_items;
        a.geo = p->geo;
        a.tl = p->tiles;
        a.grid = p->d_grid2;
        a.nx = (int)p->n_items;
        return a;
    }, [&](kp_plan p) { return p->n_items * cgroups(p, 4); }));
    KP_TRY(build_phase<BPrimal>(ps, all, bi.primal, [&](kp_plan p, int i) {
        BPrimal a{};
        a.grid = p->d_grid2;
        a.maps = p->d_maps;
        a.apod = p->d_apod;
        a.geo = p->geo;
        a.x = p->d_x;
        a.xbar = p->d_xbar;
        a.z = p->d_z;
        a.sched = p->d_sched;
        a.iter = p->d_iter;
        a.lambda = lams[i];
        a.reg = regs[i] == KP_REG_L2 ? 0 : 1;
        return a;
    }, [&](kp_plan p) { return nblk(p->geo.N, 256); }));
    KP_TRY(build_phase<BPre>(ps, l2, bi.pre, [&](kp_plan p, int) {
        BPre a{};
        a.x = p->d_xbar;
        a.maps = p->d_maps;
        a.apod = p->d_apod;
        a.geo = p->geo;
        a.grid = p->d_grid;
        return a;
    }, [&](kp_plan p) { return nblk(p->geo.G, 256); }));
    std::vector<int*> it(n);
    for (int i = 0; i < n; ++i) it[i] = ps[i]->d_iter;
    std::vector<int> boff{0, n};
    return phase_upload(bi.advance, it.data(), n * sizeof(int*), n, boff);
}

kp_status batch_interp_launch(const BatchIter& bi, cudaStream_t st) {
    const BatchPhase& ph = bi.interp;
    if (ph.nblocks == 0) return KP_OK;
    const size_t smem = (size_t)IP_CH * IpL<2>::PER_COIL * sizeof(float2);
    static PerDeviceOnce attr[3];
    KP_DISPATCH_T(bi.yt, T,
        if (attr[bi.yt].first())
            KP_TRY_CUDA(cudaFuncSetAttribute(k_interp_tile_b<2, 2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
        k_interp_tile_b<2, 2, T><<<ph.nblocks, IP_THREADS, smem, st>>>((const BInterp*)ph.d_desc, ph.d_boff, ph.ncase));
    KP_LAUNCH_CHECK();
    return KP_OK;
}

// Split-tile clearing, then the interleaved-pair spreading (variant 6: 4 warps, coil pairs).
kp_status batch_spread_launch(const BatchIter& bi, cudaStream_t st) {
    if (bi.zero.nblocks > 0) {
        k_zero_split_b<2><<<bi.zero.nblocks, 256, 0, st>>>((const BZero*)bi.zero.d_desc, bi.zero.d_boff, bi.zero.ncase);
        KP_LAUNCH_CHECK();
    }
    const BatchPhase& ph = bi.spread;
    if (ph.nblocks == 0) return KP_OK;
    static PerDeviceOnce attr;
    const size_t sm = spread_v_smem<2, 4>();
    if (attr.first())
        KP_TRY_CUDA(cudaFuncSetAttribute(k_spread_v_b<2, float2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_spread_v_b<2, float2, 4><<<ph.nblocks, 4 * 32, sm, st>>>((const BSpread*)ph.d_desc, ph.d_boff, ph.ncase);
    KP_LAUNCH_CHECK();
    return KP_OK;
}

kp_status batch_primal_launch(const BatchIter& bi, cudaStream_t st) {
    const BatchPhase& ph = bi.primal;
    if (ph.nblocks == 0) return KP_OK;
    KP_DISPATCH_T(bi.mt, MT, k_adj_primal_b<2, MT><<<ph.nblocks, 256, 0, st>>>((const BPrimal*)ph.d_desc, ph.d_boff, ph.ncase));
    KP_LAUNCH_CHECK();
    return KP_OK;
}

// Pre-step of the l2 cases' next iteration, then every case's iteration counter.
kp_status batch_pre_launch(const BatchIter& bi, cudaStream_t st) {
    const BatchPhase& ph = bi.pre;
    if (ph.nblocks > 0) {
        KP_DISPATCH_T(bi.mt, MT, k_fwd_pre_b<2, MT><<<ph.nblocks, 256, 0, st>>>((const BPre*)ph.d_desc, ph.d_boff, ph.ncase));
        KP_LAUNCH_CHECK();
    }
    k_advance_b<<<(unsigned)nblk(bi.advance.ncase, 256), 256, 0, st>>>((int* const*)bi.advance.d_desc, bi.advance.ncase);
    KP_LAUNCH_CHECK();
    return KP_OK;
}

}  // namespace kp

using namespace kp;

extern "C" {

kp_status kp_sense_forward(kp_plan plan, const void* x_dev, void* y_dev, kp_cdtype y_t, void* stream) {
    KP_RANGE("kp_sense_forward");
    if (!plan || !x_dev || !y_dev) { set_error("null argument"); return KP_EINVAL; }
    if (!plan->traj_set || (!plan->maps_set && !plan->unit_maps)) { set_error("trajectory and maps must be set"); return KP_EINVAL; }
    if (y_t != KP_C64 && y_t != KP_C32_BF16 && y_t != KP_C32_FP16) { set_error("bad y type"); return KP_EINVAL; }
    return forward_to(plan, (const float2*)x_dev, y_dev, y_t, plan->d_perm, (cudaStream_t)stream);
}

kp_status kp_sense_adjoint(kp_plan plan, const void* y_dev, kp_cdtype y_t, void* x_dev, void* stream) {
    KP_RANGE("kp_sense_adjoint");
    if (!plan || !x_dev || !y_dev) { set_error("null argument"); return KP_EINVAL; }
    if (!plan->traj_set || (!plan->maps_set && !plan->unit_maps)) { set_error("trajectory and maps must be set"); return KP_EINVAL; }
    if (y_t != KP_C64 && y_t != KP_C32_BF16 && y_t != KP_C32_FP16) { set_error("bad y type"); return KP_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    KP_TRY(adjoint_to_grid(plan, y_dev, y_t, plan->d_perm, st));
    return grid_to_image(plan, (float2*)x_dev, st);
}

}  // extern "C"
