// Internal declarations shared by the CUDA translation units of libkpdhg.
// Nothing here is part of the C ABI (include/kpdhg.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cufft.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/kpdhg.h"

namespace kp {

// A named NVTX range over a scope.  NVTX v3 is header-only and inert unless a tool (ncu,
// Nsight Systems) attaches its injection library; every entry point of the C ABI opens one
// named after itself, so a profile can select one entry point's kernels, e.g.
// ncu --nvtx --nvtx-include "kp_max_eig/" for the power method's.
struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope&) = delete;
    NvtxScope& operator=(const NvtxScope&) = delete;
};
#define KP_RANGE(name) ::kp::NvtxScope kp_nvtx_scope_(name)
// A phase of the reconstruction (preconditioner, power method, PDHG iterations) as an NVTX
// start/end range, which a filter selects regardless of the entry point it runs under
// (ncu --nvtx --nvtx-include "power_method": start/end ranges take no trailing slash).
struct NvtxPhase {
    nvtxRangeId_t id;
    explicit NvtxPhase(const char* name) : id(nvtxRangeStartA(name)) {}
    ~NvtxPhase() { nvtxRangeEnd(id); }
    NvtxPhase(const NvtxPhase&) = delete;
    NvtxPhase& operator=(const NvtxPhase&) = delete;
};
#define KP_PHASE(name) ::kp::NvtxPhase kp_nvtx_phase_(name)

// Bounds-checked build (-DKP_CHECKED, the library libkpdhg_checked.so): the hot kernels test
// each computed global-memory index against its buffer's extent before the access, skip an
// access out of range and record it: a count and the first one's site and index, in device
// words of each translation unit, which kp_bounds_report gathers and clears.  In the release
// build KP_INB is the constant true and the checks compile away.  Sites:
//   1 FFT pass load      2 FFT pass store        3 FFT pre-step image / maps / 1/Phi
//   4 interp staged row  5 interp sample I/O     6 spread own: sample values
//   7 spread own: slot   8 gather: slot read     9 gather: grid store
//  10 spread (one-phase) grid update            11 forward pre-step: image / maps / grid
//  12 adjoint combine: grid / maps / image       13 fused primal step: grid / maps / image
//  14 preconditioner: pair spectra / R          15 preconditioner: den / p
#ifdef KP_CHECKED
static __device__ unsigned int kp_oob_count;              // this translation unit's records
static __device__ unsigned long long kp_oob_first;        // site << 48 | (index mod 2^48)
__device__ __forceinline__ bool kp_in_bounds(int site, long long i, long long n) {
    if (i >= 0 && i < n) return true;
    if (atomicAdd(&kp_oob_count, 1u) == 0)
        atomicExch(&kp_oob_first, ((unsigned long long)site << 48) | ((unsigned long long)i & 0xFFFFFFFFFFFFull));
    return false;
}
#define KP_INB(site, i, n) ::kp::kp_in_bounds((site), (long long)(i), (long long)(n))
// Reads and clears this translation unit's records (after a device synchronisation).
static cudaError_t kp_oob_take(unsigned int* count, unsigned long long* first) {
    const unsigned int z = 0;
    const unsigned long long zz = 0;
    cudaError_t e = cudaMemcpyFromSymbol(count, kp_oob_count, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(first, kp_oob_first, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(kp_oob_count, &z, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(kp_oob_first, &zz, sizeof(unsigned long long));
    return e;
}
bool oob_register(cudaError_t (*take)(unsigned int*, unsigned long long*));
static const bool kp_oob_registered = oob_register(&kp_oob_take);
#else
#define KP_INB(site, i, n) true
#endif

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);

#define KP_TRY_CUDA(expr)                                                          \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            ::kp::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));   \
            return e_ == cudaErrorMemoryAllocation ? KP_ENOMEM : KP_ECUDA;         \
        }                                                                          \
    } while (0)

#define KP_TRY_CUFFT(expr)                                                         \
    do {                                                                           \
        cufftResult r_ = (expr);                                                   \
        if (r_ != CUFFT_SUCCESS) {                                                 \
            ::kp::set_error(std::string(#expr) + ": cufft error " + std::to_string((int)r_)); \
            return KP_ECUFFT;                                                      \
        }                                                                          \
    } while (0)

#define KP_TRY(expr)                                                               \
    do {                                                                           \
        kp_status s_ = (expr);                                                     \
        if (s_ != KP_OK) return s_;                                                \
    } while (0)

#define KP_LAUNCH_CHECK() KP_TRY_CUDA(cudaGetLastError())

// ---------------------------------------------------------------- geometry
constexpr int KW = 4;                // Kaiser-Bessel width supported by the kernels
constexpr int MAXD = 3;

// Geometry of one NUFFT operator, passed by value to kernels.  Arrays are indexed by
// the *active* axes 0..D-1 (slowest first); 2D problems use D = 2.
struct Geom {
    int D;
    int C;
    int64_t M;
    int n[MAXD];         // image size per axis
    int g[MAXD];         // oversampled grid size per axis
    float beta[MAXD];    // Kaiser-Bessel shape per axis
    int64_t N;           // prod n
    int64_t G;           // prod g
    float rsqrtN;        // N^{-1/2}
};

// Spreading tiles: the grid is cut into tiles of ts[d] points per axis (edge tiles smaller).
// Tiles partition the shifted index p = (i + sh) mod g of each axis, sh = ts/2, so that
// the densely sampled k-space centre (grid index 0) falls in the middle of a tile.
struct Tiles {
    int ts[MAXD];
    int nt[MAXD];        // tiles per axis
    int sh[MAXD];        // index shift
    int64_t ntiles;
};

// Grid coordinate of a sample along one axis, t = f s g / n (s = 1, or 2 on the preconditioner's
// 2N grid), evaluated in float64 as one correctly rounded quotient (f s g is exact in float64),
// so the taps and weights are those of the operator in exact arithmetic up to float32 storage
// of the offset.  Returns the first Kaiser-Bessel tap k0 = ceil(t) - W/2 (not wrapped) and sets
// *u0 = t - ceil(t) in (-1, 0]; tap j of the sample sits at distance t - (k0 + j) = u0 + W/2 - j.
__host__ __device__ __forceinline__ int grid_tap(float f, float s, int n, int g, float* u0) {
    const double t = ((double)f * (double)s * (double)g) / (double)n;
    const double c = ceil(t);
    *u0 = (float)(t - c);
    return (int)c - KW / 2;
}

// shifted tile coordinate of grid index i (0 <= i < g)
__host__ __device__ __forceinline__ int tshift(int i, int sh, int g) { int p = i + sh; return p >= g ? p - g : p; }
// grid index of shifted coordinate p (0 <= p < g)
__host__ __device__ __forceinline__ int tunshift(int p, int sh, int g) { int i = p - sh; return i < 0 ? i + g : i; }

// ---------------------------------------------------------------- float-float arithmetic
// A value held as an unevaluated sum hi + lo of two float32 numbers (about 48 significant
// bits), built from the error-free transformations of floating-point arithmetic: Knuth's
// two-sum (a + b = s + e exactly, any a, b), the fast two-sum for |a| >= |b|, and the product
// a b = p + e exactly through a fused multiply-add (Dekker's product with an FMA).  Used where
// a sum needs more than float32 (denominator sums with cancellation) and the float64 pipe of
// the GPU would be the bound.  The _rn intrinsics keep the compiler from contracting the
// additions and products whose rounding errors these formulas recover.
struct ff32 {
    float hi, lo;
};
__device__ __forceinline__ ff32 ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ff32 ff_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff32 ff_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
// (x.hi + x.lo) * b, relative error about 2^-46
__device__ __forceinline__ ff32 ff_mul(ff32 x, float b) {
    ff32 p = ff_two_prod(x.hi, b);
    return ff_fast_two_sum(p.hi, __fmaf_rn(x.lo, b, p.lo));
}
// x + y, error about 2^-46 of max(|x|, |y|)
__device__ __forceinline__ ff32 ff_add(ff32 x, ff32 y) {
    const ff32 s = ff_two_sum(x.hi, y.hi);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ double ff_to_double(ff32 x) { return (double)x.hi + (double)x.lo; }

// Once-per-device flag for host-side set-up that the runtime keeps per device, such as
// cudaFuncSetAttribute (devices 0..63): first() is true the first time it is asked on the
// current device.
struct PerDeviceOnce {
    std::atomic<unsigned long long> done{0};
    bool first() {
        int d = 0;
        cudaGetDevice(&d);
        const unsigned long long bit = 1ull << (d & 63);
        return (done.fetch_or(bit) & bit) == 0;
    }
};

// Per-device dynamic shared memory limit of one kernel whose requirement depends on the plan
// (devices 0..63): ensure() raises the limit to at least `bytes` and never lowers it, so that
// plans of different sizes can share the kernel in any order.
struct SmemLimit {
    std::atomic<int> cur[64] = {};
    template <typename F>
    cudaError_t ensure(F* fn, size_t bytes) {
        int d = 0;
        cudaError_t e = cudaGetDevice(&d);
        if (e != cudaSuccess) return e;
        std::atomic<int>& c = cur[d & 63];
        int have = c.load();
        if ((int)bytes <= have) return cudaSuccess;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        while (have < (int)bytes && !c.compare_exchange_weak(have, (int)bytes)) {}
        return cudaSuccess;
    }
};

// ---------------------------------------------------------------- complex storage helpers
__host__ __device__ inline float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline float2 cmulc(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); } // conj(a)*b

template <typename T> __device__ inline float2 ldc(const T* p, size_t i);
template <> __device__ inline float2 ldc<float2>(const float2* p, size_t i) { return p[i]; }
template <> __device__ inline float2 ldc<__half2>(const __half2* p, size_t i) { return __half22float2(p[i]); }
template <> __device__ inline float2 ldc<__nv_bfloat162>(const __nv_bfloat162* p, size_t i) { return __bfloat1622float2(p[i]); }

template <typename T> __device__ inline void stc(T* p, size_t i, float2 v);
template <> __device__ inline void stc<float2>(float2* p, size_t i, float2 v) { p[i] = v; }
template <> __device__ inline void stc<__half2>(__half2* p, size_t i, float2 v) { p[i] = __float22half2_rn(v); }
template <> __device__ inline void stc<__nv_bfloat162>(__nv_bfloat162* p, size_t i, float2 v) { p[i] = __float22bfloat162_rn(v); }

inline size_t cdtype_bytes(kp_cdtype t) { return t == KP_C64 ? 8 : 4; }

// A^H at one pixel j (row-major image index): N^{-1/2} prod_d 1/Phi_d(n_d)
// sum_c conj(s_c[j]) grid_c[n mod g] (maps == nullptr means s_c = 1).
template <int D, typename MT>
__device__ __forceinline__ float2 adj_pixel(const float2* __restrict__ grid, const MT* __restrict__ maps,
                                            const float* __restrict__ apod, const Geom& geo, int64_t j) {
    int jj[D];
    if (geo.N < ((int64_t)1 << 31)) {          // 32-bit index arithmetic (64-bit division is slow)
        unsigned r = (unsigned)j;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { jj[d] = (int)(r % (unsigned)geo.n[d]); r /= (unsigned)geo.n[d]; }
    } else {
        int64_t r = j;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { jj[d] = (int)(r % geo.n[d]); r /= geo.n[d]; }
    }
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
    if (!(KP_INB(12, j, geo.N) && KP_INB(12, gi, geo.G))) return make_float2(0.f, 0.f);
    // coils four at a time: every load of a group is issued before its products are summed
    // (the sum still runs over c = 0, 1, 2, ... in order)
    float2 acc = make_float2(0.f, 0.f);
    int c = 0;
    for (; c + 4 <= geo.C; c += 4) {
        float2 gv[4], s[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            gv[q] = grid[(size_t)(c + q) * geo.G + gi];
            s[q] = maps ? ldc<MT>(maps, (size_t)(c + q) * geo.N + j) : make_float2(1.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (maps) {
                const float2 v = cmulc(s[q], gv[q]);
                acc.x += v.x;
                acc.y += v.y;
            } else {
                acc.x += gv[q].x;
                acc.y += gv[q].y;
            }
        }
    }
    for (; c < geo.C; ++c) {
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


// Forward pre-step at one pixel: grid_c[n mod g] = s_c[j] v prod_d 1/Phi_d(n_d) for every coil.
template <int D, typename MT>
__device__ __forceinline__ void pre_pixel(float2* __restrict__ grid, const MT* __restrict__ maps,
                                          const float* __restrict__ apod, const Geom& geo, int64_t j, float2 v) {
    int jj[D];
    int64_t r = j;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) { jj[d] = (int)(r % geo.n[d]); r /= geo.n[d]; }
    int64_t gi = 0;
    float a = 1.f;
    int ao = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        int nd = jj[d] - geo.n[d] / 2;
        int id = nd < 0 ? nd + geo.g[d] : nd;
        gi = gi * geo.g[d] + id;
        a *= apod[ao + jj[d]];
        ao += geo.n[d];
    }
    if (!(KP_INB(13, j, geo.N) && KP_INB(13, gi, geo.G))) return;
    v.x *= a;
    v.y *= a;
    for (int c = 0; c < geo.C; ++c) {
        const float2 sv = maps ? ldc<MT>(maps, (size_t)c * geo.N + j) : make_float2(1.f, 0.f);
        grid[(size_t)c * geo.G + gi] = cmul(sv, v);
    }
}


// ---------------------------------------------------------------- plan
struct PrePlan;   // preconditioner workspace (kp_precond.cu)

// Device status words of a plan (d_flag[i]).
enum {
    KP_FLAG_TRAJ_BAD = 0,      // trajectory coordinates outside [-N/2, N/2] or not finite (count)
    KP_FLAG_MAX_TILE = 1,      // most own samples of a tile
    KP_FLAG_MAX_EXT = 2,       // longest spreading list of a tile
    KP_FLAG_TIMEOUT = 3,       // a bounded device wait gave up (bulk-copy staging or a grid barrier)
    KP_FLAG_PMIN = 4,          // min p as float bits
    KP_FLAG_P_BAD = 5,         // preconditioner entries not positive and finite (count)
    KP_FLAG_SCHED_BAD = 6,     // lambda_max or min p not positive and finite
    KP_FLAG_PRE_BAD = 7,       // non-positive preconditioner denominators (count)
    KP_FLAG_NONFINITE = 8,     // a solve's result holds a NaN or Inf
    KP_NFLAGS = 16
};
constexpr long long KP_DRAIN_CYCLES = 2000000000LL;   // wait for copies still in flight after a timeout

// Phases of one PDHG iteration, for event-based profiling (kp_plan_set_profiling).
enum Phase { PH_FWD_PRE = 0, PH_FFT_FWD, PH_INTERP, PH_SPREAD, PH_SPREAD_RED, PH_FFT_INV, PH_ADJ, PH_DWT_FWD,
             PH_SOFT, PH_DWT_INV, PH_EXTRAP, PH_OTHER, PH_N };

struct Graph {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    int reg = -1;            // regulariser * 4 + measurement storage type
    float lambda = -1.f;
    int64_t n_items = -1;
    int64_t launches = 0;    // own kernels per replay
};

struct Fft3Plan;                     // kp_fft.cu

}  // namespace kp

struct kp_plan_s {
    kp_params P;
    kp::Geom geo;
    kp::Tiles tiles;
    bool unit_maps = false;          // s_c = 1 (used by the preconditioner's internal plans)
    bool traj_set = false;
    bool maps_set = false;
    kp_cdtype maps_t = KP_C64;       // storage type of d_maps
    uint64_t graph_gen = 0;          // bumped whenever captured graphs become stale

    // trajectory (sorted by tile)
    float* d_t = nullptr;            // [D][M] offsets u0 = t - ceil(t) of the grid coordinates t = f g/n, sorted order
    int* d_perm = nullptr;           // sorted position -> original sample index
    int* d_key = nullptr;            // [M] cell key per original sample (scratch)
    int* d_ccnt = nullptr;           // [ncells + 1] samples per first-tap cell (then fill counters)
    int* d_coff = nullptr;           // [ncells + 1] exclusive scan of d_ccnt: first sorted position per cell
    int* d_scan_part = nullptr;      // [ncells / SCAN_B + 2] block sums of the multi-block scan
    int* d_scan_poff = nullptr;      // [ncells / SCAN_B + 2] their exclusive scan
    int64_t ncells = 0;              // ntiles x cells_per_tile
    int cells_per_tile = 0;          // prod ts_d
    int* d_cnt = nullptr;            // [ntiles + 1]
    int* d_off = nullptr;            // [ntiles + 1] exclusive scan of tile counts
    int* d_ext_off = nullptr;        // [ntiles + 1] spreading lists: offsets
    int* d_ext = nullptr;            // [M * 2^D] spreading lists: sorted sample positions
    int* d_flag = nullptr;           // [16] device status words (KP_FLAG_* below)
    int64_t max_tile = 0;
    // spreading work items: {tile, begin, end, partial slot or -1}
    int4* d_items = nullptr;
    int64_t n_items = 0, items_cap = 0;
    int* d_item_off = nullptr;       // [ntiles + 1]
    int* d_slot_off = nullptr;       // [ntiles + 1] first partial slot of each split tile
    int* d_nslots = nullptr;         // [ntiles + 1] partial slots per tile (0 = not split)
    int* d_sflag = nullptr;          // [ntiles + 1] 1 for a split tile
    int* d_spos = nullptr;           // [ntiles + 1] position of each split tile in d_split
    int* d_iitem_off = nullptr;      // [ntiles + 1] first interpolation item of each tile
    int* d_counts = nullptr;         // [8] flags and item counts for the host
    float2* d_v = nullptr;           // [D][N] TV dual variable (allocated at the first TV solve)
    float2* d_cg_r = nullptr;        // [C][M] residual of the dual conjugate gradients
    float2* d_cg_d = nullptr;        // [C][M] their search direction
    double* d_cg_trace = nullptr;    // residual norms of the last dual solve
    int64_t cg_cap = 0, cg_trace_cap = 0;
    int4* d_sort_tmp = nullptr;      // [8192] scratch of the item sort
    void* d_lsort = nullptr;         // scratch of the counting sort of longer item lists
    size_t lsort_cap = 0;
    int* d_split = nullptr;          // tiles whose list spans several work items
    int64_t n_split = 0, split_cap = 0;
    int* d_k0 = nullptr;             // [D][M] wrapped first tap ceil(t) - W/2 per sorted sample
    float* d_wt = nullptr;           // [D * W][M] Kaiser-Bessel weights per sorted sample
    int chunk = 256;                 // samples per interpolation work item (<= its block size)
    int spread_chunk = 256;          // samples per spreading work item (autotuned, multiple of 256)
    int spread_variant = 0;          // 0/3/4/5: warp-private tiles (coils x warps 4x4, 2x8, 1x8, 2x4);
                                     // 1: shared atomics, 16 coils per CTA; 2: each warp owns 4 coils;
                                     // 6/7: warp-private interleaved coil pairs, 4 coils x 4 / 8 warps;
                                     // 8/9: 3D z-plane owners; 10/11: 3D two-phase (padded tiles + gather)
    bool spread_tuned = false;
    int cluster_prox = -1;           // 2D l1 prox by one thread-block cluster: -1 unknown, 0 no, 1 yes
    int4* d_iitems = nullptr;        // interpolation work items {tile, begin, end, -1} over d_off ranges
    int64_t n_iitems = 0, iitems_cap = 0;
    // two-phase 3D spreading (variants 10, 11): own-sample items, one padded-tile slot each
    int4* d_oitems = nullptr;        // {tile, begin, end, slot} over d_off ranges, at most own_chunk samples
    int64_t n_oitems = 0, oitems_cap = 0;
    int* d_tslot = nullptr;          // [ntiles + 1] first slot of each tile
    float2* d_halo = nullptr;        // [slot][C][(TS + W - 1)^3] padded tile sums
    size_t halo_cap = 0;             // complex values allocated
    int own_chunk = 4096;

    // operator data
    void* d_maps = nullptr;          // [C][N] in maps_t storage
    float* d_apod = nullptr;         // [sum n_d] 1/Phi_d(n_d) per axis
    float2* d_grid = nullptr;        // [C][G] forward work grid
    float2* d_grid2 = nullptr;       // [C][G] adjoint (spreading) grid
    float2* d_gridF = nullptr;       // [C][G] forward grid after the FFT (d_grid keeps its zero padding)
    unsigned int* d_bar = nullptr;   // grid-barrier state of the fused kernels
    cufftHandle fft = 0;
    bool fft_ok = false;
    kp::Fft3Plan* fft3 = nullptr;    // own 3D FFT passes (kp_fft.cu) when the grid sizes allow, else cuFFT
    void* d_ystage = nullptr;        // measurements copied in from host memory (kp_pdhg_solve_host)
    size_t ystage_bytes = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copy_in = nullptr, ev_copy_done = nullptr;

    // solver state (sorted k-space order)
    float2* d_u = nullptr;           // [C][M] dual variable
    void* d_ys = nullptr;            // [C][M] sorted measurements (storage ys_t)
    kp_cdtype ys_t = KP_C64;
    float* d_ps = nullptr;           // [C][M] sorted preconditioner
    float* d_puser = nullptr;        // [C][M] preconditioner in user order (when computed here)
    float* d_f = nullptr;            // [M][D] copy of the trajectory (cycles/FOV), user order
    int traj_version = 0;
    int lists_version = -1;          // traj_version whose per-tile spreading lists d_ext / d_items hold
    float2* d_kt = nullptr;          // [C][M] scratch k-space (objective / power method)
    float2* d_x = nullptr;           // [N] primal
    float2* d_xbar = nullptr;        // [N] extrapolated primal
    float2* d_z = nullptr;           // [N] prox input / wavelet work
    float2* d_w = nullptr;           // [N] scratch image / wavelet coefficients
    float2* d_wl0 = nullptr;         // [N / 2^D] wavelet approximation ping-pong buffers
    float2* d_wl1 = nullptr;
    double* d_red = nullptr;         // [8] reductions
    float* d_sched = nullptr;        // [3 * cap] sigma, tau, theta per iteration
    double* d_schedd = nullptr;      // [4] lmax, pmin, sigma_last, tau_last
    int* d_iter = nullptr;           // iteration counter read by the captured graph
    int sched_cap = 0;

    // wavelet
    float h[8];                      // Daubechies-4 scaling filter (host copy)

    // unrolled PDHG checkpoints: per iteration xbar_k [N], u_{k+1} [C][M] (sorted), x_{k+1} [N]
    float2* d_tape = nullptr;
    size_t tape_cap = 0;
    int tape_iters = 0;
    float tape_lambda = 0.f;
    float2* d_bk = nullptr;          // [2][C][M] reverse-sweep k-space work (g_r, g_y)

    kp::Graph graphs[3];             // per regulariser
    // profiling: when on, PDHG runs without the graph and records an event at each phase
    bool profiling = false;
    cudaEvent_t* ev = nullptr;
    int* ev_phase = nullptr;
    int ev_cap = 0, ev_used = 0;
    int64_t launches = 0;            // own kernel launches issued (graph replays included)
    kp::PrePlan* pre = nullptr;
    kp_plan_s* pre_nufft = nullptr;  // NUFFT plan on the 2N image (preconditioner)
    cudaStream_t cap_stream = nullptr;
    long long wait_cycles = 2000000000LL;   // limit of every bounded device wait (SM clock cycles)
    // comparison solvers of Sec. 6 (kp_compare.cu): App. B circulant preconditioner, CG, FISTA
    float* d_circ_eig = nullptr;     // [N] eigenvalues of the circulant P (real part of the DFT of its kernel)
    float2* d_circ = nullptr;        // [N] its kernel c[k], k_d in [0, N_d)
    bool circ_ok = false;            // eigenvalues valid for the current trajectory and maps
    int circ_version = -1;
    cufftHandle fft_img = 0;         // N-point C2C on the image (circulant products)
    bool fft_img_ok = false;
    float2* d_cmp = nullptr;         // [2][N] image work vectors of CG and FISTA
    double* d_cmp_s = nullptr;       // [16] their device scalars
    double* d_cmp_trace = nullptr;   // objective trace of the last comparison solve
    int cmp_trace_cap = 0;
};

namespace kp {

// Record a phase boundary when profiling (no-op otherwise).
inline void mark(kp_plan p, int phase, cudaStream_t st) {
    if (!p->profiling || p->ev_used >= p->ev_cap) return;
    cudaEventRecord(p->ev[p->ev_used], st);
    p->ev_phase[p->ev_used] = phase;
    p->ev_used++;
}

// kp_plan.cu
kp_status plan_create_internal(kp_plan* out, const kp_params* params, bool unit_maps, cudaStream_t st);
kp_status plan_destroy_internal(kp_plan p);
kp_status set_trajectory_internal(kp_plan p, const float* traj, float traj_scale, cudaStream_t st);

// kp_nufft.cu
// A x: x [N] complex64 -> out [C][M].  Output in sorted order (perm == nullptr) or user
// order.  mode 0: plain; 1: multiply by p (sorted order); 2: PDHG dual update (uses p, y,
// sched, iter).
kp_status build_tap_tables(kp_plan p, cudaStream_t st);
kp_status forward_to(kp_plan p, const float2* x, void* out, kp_cdtype out_t, const int* perm, cudaStream_t st);
kp_status forward_dual(kp_plan p, const float2* xbar, cudaStream_t st);
// out = p (A x) in sorted order, divided by sqrt(*n2) when n2 is given (a norm kept on the device)
kp_status forward_scaled(kp_plan p, const float2* x, float2* out_sorted, const float* ps, cudaStream_t st,
                         const double* n2 = nullptr);
// A^H u: u [C][M] (sorted order if perm == nullptr, else user order) -> grid -> x.
// splits_zeroed: the split tiles' regions of d_grid2 are already zero (the fused primal kernel
// clears them after its last read of d_grid2, and solve set-up clears them once)
kp_status adjoint_to_grid(kp_plan p, const void* u, kp_cdtype u_t, const int* perm, cudaStream_t st,
                          bool splits_zeroed = false);
kp_status zero_split_only(kp_plan p, cudaStream_t st);
kp_status grid_to_image(kp_plan p, float2* x, cudaStream_t st);
kp_status autotune_spread(kp_plan p, cudaStream_t st);
kp_status adjoint_primal(kp_plan p, int reg, float lambda, cudaStream_t st);
kp_status tv_sumabs(kp_plan p, const float2* x, double* out, cudaStream_t st);
kp_status ensure_tv_dual(kp_plan p);
kp_status fill_image(float2* x, int64_t n, float2 v, cudaStream_t st);

// kp_pdhg.cu
kp_status wavelet_apply(kp_plan p, const float2* in, float2* out, bool forward, cudaStream_t st);
kp_status primal_fused(kp_plan p, int reg, float lambda, cudaStream_t st);
bool cluster_prox_ok(kp_plan p);
kp_status primal_cluster(kp_plan p, float lambda, cudaStream_t st);
kp_status solve_setup(kp_plan plan, const void* y_dev, kp_cdtype y_t, const float* p_dev, double lmax, int iters,
                      cudaStream_t st, int reg = 0, const kp_pdhg_state* start = nullptr, cudaEvent_t y_ready = nullptr);
kp_status solve_measurements(kp_plan plan, const void* y_dev, kp_cdtype y_t, cudaStream_t st);
kp_status solve_setup_a(kp_plan plan, const void* y_dev, kp_cdtype y_t, const float* p_dev, int iters, cudaStream_t st,
                        const kp_pdhg_state* start);
kp_status solve_setup_b(kp_plan plan, int iters, cudaStream_t st, int reg, const kp_pdhg_state* start);
kp_status power_begin(kp_plan p, cudaStream_t st);
kp_status power_step(kp_plan p, const float* ps_sorted, bool first, cudaStream_t st);
kp_status power_end(kp_plan p, cudaStream_t st);
kp_status pdhg_iteration(kp_plan p, int reg, float lambda, cudaStream_t st);
kp_status pdhg_iteration_concurrent(kp_plan p, int reg, float lambda, cudaStream_t st);
kp_status build_spread_items(kp_plan p, int chunk, cudaStream_t st);
kp_status build_spread_lists(kp_plan p, cudaStream_t st);
kp_status make_preconditioner_enqueue(kp_plan plan, int multichannel, float* p_dev, cudaStream_t st);
kp_status wavelet_prox_levels(kp_plan p, float lambda, cudaStream_t st);
kp_status fft_forward_only(kp_plan p, cudaStream_t st);
// In-place inverse FFT of d_grid2 (the spread grid).
kp_status fft_inverse_only(kp_plan p, cudaStream_t st);

// kp_fft.cu: own 3D FFT of all coils' grids (3D plans whose grid sizes have compiled passes;
// KPDHG_FFT=cufft at plan creation keeps cuFFT).  fft3_forward reads only the image band of `in` (zero
// elsewhere) and writes the whole spectrum to `out`; fft3_inverse works in place and leaves the
// transform valid on the image crop only.
kp_status fft3_create(kp_plan p);
void fft3_destroy(kp_plan p);
// The same passes for any batch of 3D grids (geo.C grids of geo.g points, image band geo.n per
// axis; a band as long as the axis means no pruning): fft3_make returns null when a length has
// no compiled passes.
Fft3Plan* fft3_make(const int g[3]);
void fft3_free(Fft3Plan* f);
kp_status fft3_forward_geo(const Fft3Plan* f, const Geom& g, const float2* in, float2* out, int64_t& launches,
                           cudaStream_t st);
kp_status fft3_inverse_geo(const Fft3Plan* f, const Geom& g, float2* io, int64_t& launches, cudaStream_t st);
kp_status fft3_forward(kp_plan p, const float2* in, float2* out, cudaStream_t st);
// The forward grid spectrum of image x into d_gridF, the pre-step (coil multiply, apodisation)
// formed by the first pass from x and the maps (no d_grid involved).
kp_status fft3_forward_image(kp_plan p, const float2* x, cudaStream_t st);
kp_status fft3_inverse(kp_plan p, float2* io, cudaStream_t st);
kp_status pre_only(kp_plan p, const float2* x, cudaStream_t st);
kp_status forward_grid_only(kp_plan p, const float2* x, cudaStream_t st);
kp_status interp_dual_only(kp_plan p, cudaStream_t st);
void daubechies4(float h[8]);
kp_status upload_wavelet_filter(const float h[8]);
void drop_graphs(kp_plan p);

// kp_precond.cu
void pre_destroy(kp_plan p);
kp_status circulant_enqueue(kp_plan plan, cudaStream_t st);
kp_status ensure_fft_img(kp_plan p);

// kp_compare.cu
void compare_destroy(kp_plan p);
// Reports a bounded device wait that gave up: clears the plan's timeout flag (so the report is
// consumed once), records `what` as the error message and returns KP_ETIMEOUT.
kp_status report_timeout(kp_plan p, cudaStream_t st, const char* what);

// ---------------------------------------------------------------- batched launches
// One kernel launch per phase over every case of a batch: block b of the launch belongs to the
// case c with boff[c] <= b < boff[c + 1] (boff ascending, boff[ncase] = blocks of the launch;
// a case with no blocks has boff[c] == boff[c + 1] and is never returned) and reads its
// arguments from the case's descriptor.
__device__ __forceinline__ int batch_case(const int* __restrict__ boff, int ncase, int b) {
    int lo = 0, hi = ncase - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(boff + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Device copy of one batched launch's descriptors and block offsets (owned by the batch).
struct BatchPhase {
    void* d_desc = nullptr;
    size_t desc_cap = 0;
    int* d_boff = nullptr;
    size_t boff_cap = 0;
    int ncase = 0;
    unsigned nblocks = 0;
};
kp_status phase_upload(BatchPhase& ph, const void* descs, size_t desc_bytes, int ncase, const std::vector<int>& boff);
void phase_free(BatchPhase& ph);

// The batched 2D PDHG iteration (l2 and l1-wavelet cases; every case shares the dimension, the
// k-space storage type and the maps storage type).  Built outside stream capture (descriptors
// are uploaded with blocking copies), launched inside it.
struct BatchIter {
    BatchPhase interp, zero, spread, primal, pre, advance;
    std::vector<BatchPhase> fwd, inv;    // wavelet levels 0 .. Lmax-1 (forward), same (inverse)
    kp_cdtype yt = KP_C64, mt = KP_C64;
    bool built = false;
};
void batch_iter_free(BatchIter& bi);
// NUFFT-side phases (interpolation + dual step, split-tile clearing, spreading, primal step,
// pre-step of the l2 cases, iteration counters).
kp_status batch_nufft_build(const std::vector<kp_plan>& ps, const std::vector<int>& regs,
                            const std::vector<float>& lams, BatchIter& bi);
kp_status batch_interp_launch(const BatchIter& bi, cudaStream_t st);
kp_status batch_spread_launch(const BatchIter& bi, cudaStream_t st);
kp_status batch_primal_launch(const BatchIter& bi, cudaStream_t st);
kp_status batch_pre_launch(const BatchIter& bi, cudaStream_t st);
// Wavelet prox of the l1 cases: forward levels then inverse levels (level 0 also extrapolates
// and writes the next forward grid), one launch per level over the cases that have it.
kp_status batch_wavelet_build(const std::vector<kp_plan>& ps, const std::vector<int>& regs,
                              const std::vector<float>& lams, BatchIter& bi);
kp_status batch_wavelet_launch(const BatchIter& bi, cudaStream_t st);

}  // namespace kp
