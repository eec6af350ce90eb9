// Plan life cycle, trajectory binning (counting sort by grid tile) and coil maps.
//
// The trajectory step converts each sample to grid coordinates t_d = f_d * (g_d / n_d)
// (float64, Sec. 6 NUFFT with oversampling g/n; kept as the first tap and a float32 offset),
// sorts samples by the grid tile that
// holds their first Kaiser-Bessel tap, and builds, per tile, the list of samples whose
// W^D footprint touches that tile (used by the spreading kernel, which owns one output
// tile per CTA and therefore needs no global atomics and no zero-fill of the grid).
#include "kp_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace kp {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

#ifdef KP_CHECKED
// The translation units' record readers (registered during static initialisation).
static std::vector<cudaError_t (*)(unsigned int*, unsigned long long*)>& oob_readers() {
    static std::vector<cudaError_t (*)(unsigned int*, unsigned long long*)> r;
    return r;
}
bool oob_register(cudaError_t (*take)(unsigned int*, unsigned long long*)) {
    oob_readers().push_back(take);
    return true;
}
#endif

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ int wrap(int k, int g) { return k < 0 ? k + g : (k >= g ? k - g : k); }

// Single-CTA exclusive scan of n ints: out[0..n] (out[n] = total).
__global__ void k_scan_excl(const int* __restrict__ in, int* __restrict__ out, int64_t n) {
    __shared__ long long part[1024];
    const int T = blockDim.x;
    const int64_t per = (n + T - 1) / T;
    const int64_t beg = (int64_t)threadIdx.x * per;
    const int64_t end = beg + per < n ? beg + per : n;
    long long s = 0;
    for (int64_t i = beg; i < end; ++i) s += in[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        long long v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    long long run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int64_t i = beg; i < end; ++i) {
        out[i] = (int)run;
        run += in[i];
    }
    if (threadIdx.x == T - 1) out[n] = (int)part[T - 1];
}

// Exclusive scan of n ints over many CTAs: k_scan_part sums each block of SCAN_B elements,
// the block sums are scanned by k_scan_excl, and k_scan_fin scans each block from its offset.
// out[n] = total.
constexpr int SCAN_T = 256, SCAN_PER = 8, SCAN_B = SCAN_T * SCAN_PER;

__device__ __forceinline__ int block_excl_scan(int v, int* total) {
    __shared__ int ws[SCAN_T / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < SCAN_T / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < SCAN_T / 32) ws[lane] = t;
    }
    __syncthreads();
    const int before = w ? ws[w - 1] : 0;
    *total = ws[SCAN_T / 32 - 1];
    return before + x - v;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_part(const int* __restrict__ in, int64_t n, int* __restrict__ part) {
    const int64_t b0 = (int64_t)blockIdx.x * SCAN_B + (int64_t)threadIdx.x * SCAN_PER;
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) s += b0 + k < n ? in[b0 + k] : 0;
    int tot;
    (void)block_excl_scan(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_fin(const int* __restrict__ in, int64_t n, const int* __restrict__ part_off,
                                                     int* __restrict__ out) {
    const int64_t b0 = (int64_t)blockIdx.x * SCAN_B + (int64_t)threadIdx.x * SCAN_PER;
    int v[SCAN_PER], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) { v[k] = b0 + k < n ? in[b0 + k] : 0; s += v[k]; }
    int tot;
    int run = block_excl_scan(s, &tot) + part_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        if (b0 + k < n) out[b0 + k] = run;
        run += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = part_off[gridDim.x];
}

// Tile index of one sample from its first taps k0 (already wrapped into [0, g)).
template <int D>
__device__ __forceinline__ int64_t tile_of(const int* k0w, const Tiles& tl) {
    int64_t key = 0;
    for (int d = 0; d < D; ++d) key = key * tl.nt[d] + k0w[d] / tl.ts[d];
    return key;   // k0w already shifted
}

// Pass 1: validate, convert to grid coordinates, key by the first tap's grid cell in tile-major
// order (tile index x cells per tile + the cell's local index, slowest axis first), histogram.
template <int D>
__global__ void k_traj_key(const float* __restrict__ traj, float traj_scale, Geom geo, Tiles tl, int cells_per_tile,
                           int* __restrict__ key, int* __restrict__ cnt, int* __restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= geo.M) return;
    int64_t tile = 0, cell = 0;
    bool bad = false;
    for (int d = 0; d < D; ++d) {
        float f = traj[i * D + d];
        float half = 0.5f * (float)geo.n[d];
        if (!(f * traj_scale >= -half && f * traj_scale <= half)) bad = true;   // also catches NaN
        float u0;
        const int k0 = grid_tap(bad ? 0.f : f, traj_scale, geo.n[d], geo.g[d], &u0);
        const int pd = tshift(wrap(k0, geo.g[d]), tl.sh[d], geo.g[d]);
        const int td = pd / tl.ts[d];
        tile = tile * tl.nt[d] + td;
        cell = cell * tl.ts[d] + (pd - td * tl.ts[d]);
    }
    if (bad) atomicAdd(flag, 1);
    const int64_t kk = tile * cells_per_tile + cell;
    key[i] = (int)kk;
    atomicAdd(&cnt[kk], 1);
}

// Tile ranges of the cell-sorted order: off[t] = first sorted position of tile t (t <= ntiles).
__global__ void k_tile_off(const int* __restrict__ coff, int64_t ntiles, int cells_per_tile, int* __restrict__ off,
                           int* __restrict__ cnt) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    off[t] = coff[t * cells_per_tile];
    if (t < ntiles) cnt[t] = coff[(t + 1) * cells_per_tile] - coff[t * cells_per_tile];
}

// Pass 2: scatter sample i to its slot in the sorted order, with its wrapped first tap
// k0t[d][pos] and its float32 offset u0[d][pos] = t - ceil(t) (grid_tap).
template <int D>
__global__ void k_traj_scatter(const float* __restrict__ traj, float traj_scale, Geom geo,
                               const int* __restrict__ key, const int* __restrict__ off,
                               int* __restrict__ fill, int* __restrict__ perm, float* __restrict__ u0t,
                               int* __restrict__ k0t) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= geo.M) return;
    int kk = key[i];
    int pos = off[kk] + atomicAdd(&fill[kk], 1);
    perm[pos] = (int)i;
    for (int d = 0; d < D; ++d) {
        float f = traj[i * D + d];
        float half = 0.5f * (float)geo.n[d];
        if (!(f * traj_scale >= -half && f * traj_scale <= half)) f = 0.f;
        float u0;
        const int k0 = grid_tap(f, traj_scale, geo.n[d], geo.g[d], &u0);
        u0t[(int64_t)d * geo.M + pos] = u0;
        k0t[(int64_t)d * geo.M + pos] = wrap(k0, geo.g[d]);
    }
}

// Tiles touched by the footprint of sorted sample s, per axis (1 or 2 each).
template <int D>
__device__ __forceinline__ void footprint_tiles(const int* __restrict__ k0t, int64_t s, const Geom& geo,
                                                const Tiles& tl, int lo[D], int hi[D]) {
    for (int d = 0; d < D; ++d) {
        const int k0 = k0t[(int64_t)d * geo.M + s];
        int a = tshift(k0, tl.sh[d], geo.g[d]);
        int b = tshift(wrap(k0 + KW - 1, geo.g[d]), tl.sh[d], geo.g[d]);
        lo[d] = a / tl.ts[d];
        hi[d] = b / tl.ts[d];
    }
}

template <int D, bool FILL>
__global__ void k_ext(const int* __restrict__ k0t, Geom geo, Tiles tl, int* __restrict__ cnt,
                      const int* __restrict__ off, int* __restrict__ ext) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= geo.M) return;
    int lo[D], hi[D];
    footprint_tiles<D>(k0t, s, geo, tl, lo, hi);
    for (int m = 0; m < (1 << D); ++m) {
        int64_t key = 0;
        bool dup = false;
        for (int d = 0; d < D; ++d) {
            int bit = (m >> (D - 1 - d)) & 1;
            if (bit && hi[d] == lo[d]) dup = true;
            key = key * tl.nt[d] + (bit ? hi[d] : lo[d]);
        }
        if (dup) continue;
        if (FILL) {
            int pos = off[key] + atomicAdd(&cnt[key], 1);
            ext[pos] = (int)s;
        } else {
            atomicAdd(&cnt[key], 1);
        }
    }
}

__global__ void k_max_count(const int* __restrict__ cnt, int64_t n, int* __restrict__ out) {
    int m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, cnt[i]);
    atomicMax(out, m);
}

// Spreading work items: each tile's list is cut into chunks of at most `chunk` samples;
// tiles with more than one chunk get partial slots.  Empty tiles still get one item so
// that their (zero) grid values are written.
__global__ void k_chunks(const int* __restrict__ ext_off, int64_t ntiles, int chunk, int* __restrict__ nch,
                         int* __restrict__ nsl) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    int cnt = ext_off[t + 1] - ext_off[t];
    int nc = cnt <= chunk ? 1 : (cnt + chunk - 1) / chunk;
    nch[t] = nc;
    nsl[t] = nc > 1 ? nc : 0;
}

__global__ void k_ichunks(const int* __restrict__ off, int64_t ntiles, int chunk, int* __restrict__ nch) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const int cnt = off[t + 1] - off[t];
    nch[t] = (cnt + chunk - 1) / chunk;
}

__global__ void k_iitems(const int* __restrict__ off, const int* __restrict__ item_off, int64_t ntiles, int chunk,
                         int4* __restrict__ items) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const int beg = off[t], end = off[t + 1];
    const int nc = item_off[t + 1] - item_off[t];
    for (int k = 0; k < nc; ++k) {
        const int b = beg + k * chunk;
        const int e = b + chunk < end ? b + chunk : end;
        items[item_off[t] + k] = make_int4((int)t, b, e, -1);
    }
}

__global__ void k_slot_ids(int4* __restrict__ items, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) items[i].w = (int)i;
}

__global__ void k_items(const int* __restrict__ ext_off, const int* __restrict__ item_off,
                        const int* __restrict__ slot_off, const int* __restrict__ nsl, int64_t ntiles, int chunk,
                        int4* __restrict__ items) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    int beg = ext_off[t], end = ext_off[t + 1];
    int nc = item_off[t + 1] - item_off[t];
    for (int k = 0; k < nc; ++k) {
        int b = beg + k * chunk;
        int e = b + chunk < end ? b + chunk : end;
        items[item_off[t] + k] = make_int4((int)t, b, e, nsl[t] > 0 ? slot_off[t] + k : -1);
    }
}

// Split tiles (tiles with partial slots) in tile order: f[t] = 1 for a split tile; the exclusive
// scan of f gives each its position in the list.
__global__ void k_split_flags(const int* __restrict__ nsl, int64_t ntiles, int* __restrict__ f) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntiles) f[t] = nsl[t] > 0 ? 1 : 0;
}

__global__ void k_split_list(const int* __restrict__ nsl, const int* __restrict__ pos, int64_t ntiles,
                             int* __restrict__ split) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntiles && nsl[t] > 0) split[pos[t]] = (int)t;
}

// Everything the host needs after binning, in one array for one copy: the four trajectory
// flags, then the numbers of spreading items, split tiles, interpolation items and own items.
__global__ void k_gather_counts(const int* __restrict__ flag, const int* __restrict__ n_items,
                                const int* __restrict__ n_split, const int* __restrict__ n_iitems,
                                const int* __restrict__ n_oitems, int* __restrict__ out) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < 4; ++i) out[i] = flag[i];
        out[4] = *n_items;
        out[5] = *n_split;
        out[6] = *n_iitems;
        out[7] = *n_oitems;
    }
}

// Longest-first order of at most SORT_MAX work items (length z - y descending; equal lengths
// keep their index order, as a stable sort would): one CTA sorts the keys
// (2^18 - 1 - length) * 2^13 + index bitonically in shared memory, then out[i] = in[index of
// the i-th key].
constexpr int SORT_MAX = 8192;
__global__ void __launch_bounds__(1024) k_sort_items(const int4* __restrict__ in, int n, int4* __restrict__ out) {
    __shared__ unsigned key[SORT_MAX];
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        if (i < n) {
            const int len = max(0, min(in[i].z - in[i].y, (1 << 18) - 1));
            key[i] = ((unsigned)((1 << 18) - 1 - len) << 13) | (unsigned)i;
        } else {
            key[i] = 0xFFFFFFFFu;
        }
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned a = key[i], b = key[ixj];
                    if ((a > b) == ((i & k) == 0)) {
                        key[i] = b;
                        key[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = in[key[i] & 0x1FFFu];
}

template <typename T>
__global__ void k_copy_maps(const T* __restrict__ in, T* __restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------- host helpers
static double kb_apod_host(double n, double g, double beta) {
    // Fourier transform of the Kaiser-Bessel window at frequency n/g (width KW).
    const double pi = 3.14159265358979323846;
    double z2 = beta * beta - (pi * KW * n / g) * (pi * KW * n / g);
    if (z2 > 0) { double z = std::sqrt(z2); return KW * std::sinh(z) / z; }
    if (z2 < 0) { double z = std::sqrt(-z2); return KW * std::sin(z) / z; }
    return KW;
}

template <typename T>
static kp_status alloc(T** p, size_t count) {
    KP_TRY_CUDA(cudaMalloc((void**)p, count * sizeof(T) > 0 ? count * sizeof(T) : 16));
    return KP_OK;
}

kp_status plan_create_internal(kp_plan* out, const kp_params* prm, bool unit_maps, cudaStream_t st) {
    if (!out || !prm) { set_error("null argument"); return KP_EINVAL; }
    *out = nullptr;
    const int D = prm->ndim;
    if (D != 2 && D != 3) { set_error("ndim must be 2 or 3"); return KP_EINVAL; }
    if (prm->ncoils < 1 || prm->nsamples < 1) { set_error("ncoils and nsamples must be >= 1"); return KP_EINVAL; }
    if (prm->nsamples > (int64_t)1 << 26) { set_error("nsamples too large (max 2^26)"); return KP_EINVAL; }
    if (prm->kernel_width != KW) { set_error("kernel_width must be 4"); return KP_EINVAL; }
    if (!(prm->oversamp >= 1.0f && prm->oversamp <= 4.0f)) { set_error("oversamp must be in [1, 4]"); return KP_EINVAL; }
    if (prm->wavelet_levels < 0 || prm->wavelet_levels > 10) { set_error("wavelet_levels out of range"); return KP_EINVAL; }
    for (int d = 0; d < D; ++d) {
        if (prm->img[d] < 8 || prm->img[d] > 4096) { set_error("image sizes must be in [8, 4096]"); return KP_EINVAL; }
        if (prm->wavelet_levels > 0 && (prm->img[d] % (1LL << prm->wavelet_levels)) != 0) {
            set_error("every image size must be divisible by 2^wavelet_levels"); return KP_EINVAL;
        }
    }
    kp_plan p = new (std::nothrow) kp_plan_s();
    if (!p) { set_error("host allocation failed"); return KP_ENOMEM; }
    p->P = *prm;
    p->unit_maps = unit_maps;
    Geom& g = p->geo;
    g.D = D;
    g.C = prm->ncoils;
    g.M = prm->nsamples;
    g.N = 1;
    g.G = 1;
    for (int d = 0; d < MAXD; ++d) { g.n[d] = 1; g.g[d] = 1; g.beta[d] = 0.f; }
    for (int d = 0; d < D; ++d) {
        int n = (int)prm->img[d];
        int gg = (int)std::ceil((double)prm->oversamp * n - 1e-9);
        gg += gg & 1;
        g.n[d] = n;
        g.g[d] = gg;
        double a = (double)gg / n;
        double b2 = (KW / a) * (KW / a) * (a - 0.5) * (a - 0.5) - 0.8;
        if (b2 <= 0) { delete p; set_error("oversampling too small for a Kaiser-Bessel width of 4"); return KP_EINVAL; }
        g.beta[d] = (float)(3.14159265358979323846 * std::sqrt(b2));
        g.N *= n;
        g.G *= gg;
    }
    g.rsqrtN = (float)(1.0 / std::sqrt((double)g.N));
    if ((int64_t)g.C * g.G > ((int64_t)1 << 34)) { delete p; set_error("grid too large"); return KP_EINVAL; }
    Tiles& tl = p->tiles;
    tl.ntiles = 1;
    for (int d = 0; d < MAXD; ++d) { tl.ts[d] = 1; tl.nt[d] = 1; tl.sh[d] = 0; }
    for (int d = 0; d < D; ++d) {
        // Tile edge: the largest size <= 16 (2D) / 8 (3D) whose last, ragged tile still has at
        // least W - 1 points, so a footprint of W consecutive grid points (with wrap-around)
        // touches at most two tiles per axis.
        const int base = D == 2 ? 16 : 8, lo = D == 2 ? 8 : 4;
        int ts = g.g[d];
        if (g.g[d] > base) {
            for (int c = base; c >= lo; --c) {
                const int r = g.g[d] % c;
                if (r == 0 || r >= KW - 1) { ts = c; break; }
            }
        }
        tl.ts[d] = ts;
        tl.sh[d] = ts < g.g[d] ? ts / 2 : 0;
        tl.nt[d] = (g.g[d] + tl.ts[d] - 1) / tl.ts[d];
        tl.ntiles *= tl.nt[d];
    }
    kp::daubechies4(p->h);
    {
        kp_status fs = upload_wavelet_filter(p->h);
        if (fs != KP_OK) { delete p; return fs; }
    }

    const int64_t C = g.C, M = g.M, N = g.N, G = g.G;
    kp_status s = KP_OK;
#define KP_A(ptr, cnt) do { s = alloc(&(ptr), (size_t)(cnt)); if (s != KP_OK) { plan_destroy_internal(p); return s; } } while (0)
    KP_A(p->d_t, (size_t)D * M);
    KP_A(p->d_f, (size_t)D * M);
    KP_A(p->d_perm, M);
    KP_A(p->d_key, M);
    KP_A(p->d_cnt, tl.ntiles + 1);
    p->cells_per_tile = 1;
    for (int d = 0; d < D; ++d) p->cells_per_tile *= tl.ts[d];
    p->ncells = tl.ntiles * p->cells_per_tile;
    if (p->ncells >= ((int64_t)1 << 31) - 1) { plan_destroy_internal(p); set_error("grid too large for the cell sort"); return KP_EINVAL; }
    KP_A(p->d_ccnt, p->ncells + 1);
    KP_A(p->d_coff, p->ncells + 1);
    KP_A(p->d_scan_part, p->ncells / SCAN_B + 2);
    KP_A(p->d_scan_poff, p->ncells / SCAN_B + 2);
    KP_A(p->d_off, tl.ntiles + 1);
    KP_A(p->d_ext_off, tl.ntiles + 1);
    KP_A(p->d_ext, (size_t)M << D);
    KP_A(p->d_item_off, tl.ntiles + 1);
    KP_A(p->d_k0, (size_t)D * M);
    KP_A(p->d_wt, (size_t)D * KW * M);
    KP_A(p->d_slot_off, tl.ntiles + 1);
    KP_A(p->d_nslots, tl.ntiles + 1);
    KP_A(p->d_flag, KP_NFLAGS);
    {
        float* ap = nullptr;
        int tot = 0;
        for (int d = 0; d < D; ++d) tot += g.n[d];
        KP_A(ap, tot);
        p->d_apod = ap;
        std::vector<float> h(tot);
        int o = 0;
        for (int d = 0; d < D; ++d) {
            for (int j = 0; j < g.n[d]; ++j) {
                double nn = (double)(j - g.n[d] / 2);
                h[o + j] = (float)(1.0 / kb_apod_host(nn, g.g[d], g.beta[d]));
            }
            o += g.n[d];
        }
        KP_TRY_CUDA(cudaMemcpy(ap, h.data(), tot * sizeof(float), cudaMemcpyHostToDevice));
    }
    if (!unit_maps) {
        char* mp = nullptr;
        KP_A(mp, (size_t)C * N * 8);
        p->d_maps = mp;
    }
    KP_A(p->d_grid, (size_t)C * G);
    KP_A(p->d_grid2, (size_t)C * G);
    KP_A(p->d_gridF, (size_t)C * G);
    KP_A(p->d_bar, 4);
    KP_TRY_CUDA(cudaMemset(p->d_bar, 0, 4 * sizeof(unsigned int)));
    KP_A(p->d_u, (size_t)C * M);
    {
        char* yp = nullptr;
        KP_A(yp, (size_t)C * M * 8);
        p->d_ys = yp;
    }
    KP_A(p->d_ps, (size_t)C * M);
    KP_A(p->d_puser, (size_t)C * M);
    KP_A(p->d_kt, (size_t)C * M);
    KP_A(p->d_x, N);
    KP_A(p->d_xbar, N);
    KP_A(p->d_z, N);
    KP_A(p->d_w, N);
    if (prm->wavelet_levels > 0) {
        KP_A(p->d_wl0, (N >> D) + 1);
        KP_A(p->d_wl1, (N >> D) + 1);
    }
    KP_A(p->d_red, 16);
    KP_A(p->d_sflag, tl.ntiles + 1);
    KP_A(p->d_spos, tl.ntiles + 1);
    KP_A(p->d_iitem_off, tl.ntiles + 1);
    KP_A(p->d_tslot, tl.ntiles + 1);
    KP_A(p->d_counts, 8);
    KP_A(p->d_schedd, 8);
    KP_A(p->d_iter, 4);
#undef KP_A
    int dims[3] = {g.g[0], g.g[1], g.g[2]};
    cufftResult fr = cufftPlanMany(&p->fft, D, dims, nullptr, 1, (int)G, nullptr, 1, (int)G, CUFFT_C2C, (int)C);
    if (fr != CUFFT_SUCCESS) {
        plan_destroy_internal(p);
        set_error("cufftPlanMany failed: " + std::to_string((int)fr));
        return fr == CUFFT_ALLOC_FAILED ? KP_ENOMEM : KP_ECUFFT;
    }
    p->fft_ok = true;
    {
        const kp_status fs = fft3_create(p);
        if (fs != KP_OK) { plan_destroy_internal(p); return fs; }
    }
    if (cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        plan_destroy_internal(p);
        set_error("cudaStreamCreate failed");
        return KP_ECUDA;
    }
    (void)st;
    *out = p;
    return KP_OK;
}

kp_status plan_destroy_internal(kp_plan p) {
    if (!p) return KP_OK;
    cudaDeviceSynchronize();
    drop_graphs(p);
    pre_destroy(p);
    compare_destroy(p);
    if (p->fft_ok) cufftDestroy(p->fft);
    fft3_destroy(p);
    void* bufs[] = {p->d_t, p->d_f, p->d_perm, p->d_key, p->d_ccnt, p->d_coff, p->d_scan_part, p->d_scan_poff, p->d_cnt, p->d_off, p->d_ext_off, p->d_ext, p->d_flag,
                    p->d_items, p->d_iitems, p->d_item_off, p->d_slot_off, p->d_nslots, p->d_split, p->d_k0, p->d_wt,
                    p->d_grid2, p->d_gridF, p->d_bar, p->d_tape, p->d_bk,
                    p->d_maps, p->d_apod, p->d_grid, p->d_u, p->d_ys, p->d_ps, p->d_puser, p->d_kt,
                    p->d_x, p->d_xbar, p->d_z, p->d_w, p->d_wl0, p->d_wl1, p->d_red, p->d_sched, p->d_schedd, p->d_iter,
                    p->d_oitems, p->d_tslot, p->d_halo, p->d_sflag, p->d_spos, p->d_iitem_off, p->d_counts,
                    p->d_sort_tmp, p->d_lsort, p->d_v, p->d_cg_r, p->d_cg_d, p->d_cg_trace};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    if (p->ev_copy_in) cudaEventDestroy(p->ev_copy_in);
    if (p->ev_copy_done) cudaEventDestroy(p->ev_copy_done);
    if (p->d_ystage) cudaFree(p->d_ystage);
    for (int i = 0; i < p->ev_cap; ++i) cudaEventDestroy(p->ev[i]);
    delete[] p->ev;
    delete[] p->ev_phase;
    delete p;
    return KP_OK;
}

// Reorders work items longest first, so the CTAs that take longest start in the first wave
// instead of forming a tail; items are independent, so the order is free.  Up to SORT_MAX items:
// one CTA's bitonic sort (stable); longer lists: a counting sort by length on the device
// (lengths are at most the item size), equal lengths in any order.
__global__ void k_len_hist(const int4* __restrict__ items, int64_t n, int maxlen, int* __restrict__ hist) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int len = max(0, min(items[i].z - items[i].y, maxlen));
    atomicAdd(&hist[maxlen - len], 1);                    // bucket 0 holds the longest items
}

__global__ void k_len_scatter(const int4* __restrict__ items, int64_t n, int maxlen, const int* __restrict__ off,
                              int* __restrict__ fill, int4* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 it = items[i];
    const int b = maxlen - max(0, min(it.z - it.y, maxlen));
    out[off[b] + atomicAdd(&fill[b], 1)] = it;
}

static kp_status sort_items_longest_first(kp_plan p, int4* d_items, int64_t n, int maxlen, cudaStream_t st) {
    if (n <= 1) return KP_OK;
    if (n <= SORT_MAX) {
        if (!p->d_sort_tmp) KP_TRY_CUDA(cudaMalloc(&p->d_sort_tmp, SORT_MAX * sizeof(int4)));
        k_sort_items<<<1, 1024, 0, st>>>(d_items, (int)n, p->d_sort_tmp);
        KP_LAUNCH_CHECK();
        KP_TRY_CUDA(cudaMemcpyAsync(d_items, p->d_sort_tmp, n * sizeof(int4), cudaMemcpyDeviceToDevice, st));
        p->launches += 1;
        return KP_OK;
    }
    // scratch: the sorted copy, then the length histogram, its scan and the fill counters
    const size_t need = (size_t)n * sizeof(int4) + 3 * (size_t)(maxlen + 2) * sizeof(int);
    if (need > p->lsort_cap) {
        if (p->d_lsort) cudaFree(p->d_lsort);
        p->d_lsort = nullptr;
        p->lsort_cap = 0;
        KP_TRY_CUDA(cudaMalloc(&p->d_lsort, need));
        p->lsort_cap = need;
    }
    int4* out = (int4*)p->d_lsort;
    int* hist = (int*)(out + n);
    int* off = hist + (maxlen + 2);
    int* fill = off + (maxlen + 2);
    KP_TRY_CUDA(cudaMemsetAsync(hist, 0, (size_t)(maxlen + 2) * sizeof(int), st));
    KP_TRY_CUDA(cudaMemsetAsync(fill, 0, (size_t)(maxlen + 2) * sizeof(int), st));
    k_len_hist<<<nblk(n, 256), 256, 0, st>>>(d_items, n, maxlen, hist);
    k_scan_excl<<<1, 1024, 0, st>>>(hist, off, maxlen + 1);
    k_len_scatter<<<nblk(n, 256), 256, 0, st>>>(d_items, n, maxlen, off, fill, out);
    KP_LAUNCH_CHECK();
    KP_TRY_CUDA(cudaMemcpyAsync(d_items, out, n * sizeof(int4), cudaMemcpyDeviceToDevice, st));
    p->launches += 3;
    return KP_OK;
}

// Spreading work items: each tile's list cut into pieces of at most `chunk` samples (a
// multiple of the kernels' staging size); tiles cut into several pieces are "split" and
// accumulate with global atomics into a region cleared before each spread.  The counts are
// enqueued first (d_item_off[ntiles] items, d_spos[ntiles] split tiles); the items are built
// once the host knows them.
static void spread_items_counts(kp_plan p, int chunk, cudaStream_t st) {
    const Tiles& tl = p->tiles;
    const unsigned tb = nblk(tl.ntiles, 256);
    k_chunks<<<tb, 256, 0, st>>>(p->d_ext_off, tl.ntiles, chunk, p->d_cnt, p->d_nslots);
    k_scan_excl<<<1, 1024, 0, st>>>(p->d_cnt, p->d_item_off, tl.ntiles);
    k_scan_excl<<<1, 1024, 0, st>>>(p->d_nslots, p->d_slot_off, tl.ntiles);
    k_split_flags<<<tb, 256, 0, st>>>(p->d_nslots, tl.ntiles, p->d_sflag);
    k_scan_excl<<<1, 1024, 0, st>>>(p->d_sflag, p->d_spos, tl.ntiles);
    p->launches += 5;
}

static kp_status spread_items_finish(kp_plan p, int chunk, int64_t n_items, int64_t n_split, cudaStream_t st) {
    const Tiles& tl = p->tiles;
    const unsigned tb = nblk(tl.ntiles, 256);
    p->spread_chunk = chunk;
    p->n_items = n_items;
    if (p->n_items > p->items_cap) {
        if (p->d_items) cudaFree(p->d_items);
        p->d_items = nullptr;
        KP_TRY_CUDA(cudaMalloc(&p->d_items, p->n_items * sizeof(int4)));
        p->items_cap = p->n_items;
    }
    p->n_split = n_split;
    if (p->n_split > p->split_cap) {
        if (p->d_split) cudaFree(p->d_split);
        p->d_split = nullptr;
        KP_TRY_CUDA(cudaMalloc(&p->d_split, p->n_split * sizeof(int)));
        p->split_cap = p->n_split;
    }
    if (p->n_split > 0) k_split_list<<<tb, 256, 0, st>>>(p->d_nslots, p->d_spos, tl.ntiles, p->d_split);
    k_items<<<tb, 256, 0, st>>>(p->d_ext_off, p->d_item_off, p->d_slot_off, p->d_nslots, tl.ntiles, chunk, p->d_items);
    KP_LAUNCH_CHECK();
    p->launches += 2;
    return sort_items_longest_first(p, p->d_items, p->n_items, chunk, st);
}

// The four trajectory flags and the item counts into d_counts, read with one copy.
static kp_status read_counts(kp_plan p, const int* n_iitems, const int* n_oitems, int out[8], cudaStream_t st) {
    const int64_t nt = p->tiles.ntiles;
    k_gather_counts<<<1, 32, 0, st>>>(p->d_flag, p->d_item_off + nt, p->d_spos + nt, n_iitems, n_oitems, p->d_counts);
    KP_LAUNCH_CHECK();
    p->launches += 1;
    KP_TRY_CUDA(cudaMemcpyAsync(out, p->d_counts, 8 * sizeof(int), cudaMemcpyDeviceToHost, st));
    KP_TRY_CUDA(cudaStreamSynchronize(st));
    return KP_OK;
}

// Rebuilds the spreading items for another chunk size (the autotuner's candidates).
kp_status build_spread_items(kp_plan p, int chunk, cudaStream_t st) {
    drop_graphs(p);
    spread_items_counts(p, chunk, st);
    KP_LAUNCH_CHECK();
    int cnt[8];
    KP_TRY(read_counts(p, p->d_item_off + p->tiles.ntiles, p->d_item_off + p->tiles.ntiles, cnt, st));
    return spread_items_finish(p, chunk, cnt[4], cnt[5], st);
}

// Own-sample items of the two-phase spreading: each tile's own samples (those whose first tap
// lies in it) cut into pieces of at most own_chunk; item i writes padded-tile slot i, and
// d_tslot[t] is the first slot of tile t (d_tslot[ntiles] items).  The slot storage itself is
// allocated on first use.
static void own_items_counts(kp_plan p, cudaStream_t st) {
    const Tiles& tl = p->tiles;
    const unsigned tb = nblk(tl.ntiles, 256);
    p->own_chunk = p->geo.D == 2 ? 512 : 4096;   // 2D grids have few tiles: shorter items spread the work
    k_ichunks<<<tb, 256, 0, st>>>(p->d_off, tl.ntiles, p->own_chunk, p->d_cnt);
    k_scan_excl<<<1, 1024, 0, st>>>(p->d_cnt, p->d_tslot, tl.ntiles);
    p->launches += 2;
}

static kp_status own_items_finish(kp_plan p, int64_t n, cudaStream_t st) {
    const Tiles& tl = p->tiles;
    const unsigned tb = nblk(tl.ntiles, 256);
    p->n_oitems = n;
    if (p->n_oitems > p->oitems_cap) {
        if (p->d_oitems) cudaFree(p->d_oitems);
        p->d_oitems = nullptr;
        KP_TRY_CUDA(cudaMalloc(&p->d_oitems, p->n_oitems * sizeof(int4)));
        p->oitems_cap = p->n_oitems;
    }
    if (p->n_oitems > 0) {
        k_iitems<<<tb, 256, 0, st>>>(p->d_off, p->d_tslot, tl.ntiles, p->own_chunk, p->d_oitems);
        KP_LAUNCH_CHECK();
        k_slot_ids<<<nblk(p->n_oitems, 256), 256, 0, st>>>(p->d_oitems, p->n_oitems);
        KP_LAUNCH_CHECK();
        p->launches += 2;
        KP_TRY(sort_items_longest_first(p, p->d_oitems, p->n_oitems, p->own_chunk, st));   // slot ids travel with the items
    }
    return KP_OK;
}

// Per-tile lists of the sorted samples whose footprint touches the tile (d_ext_off, d_ext; the
// longest list's length in d_flag[KP_FLAG_MAX_EXT]).
static void spread_lists_enqueue(kp_plan p, cudaStream_t st) {
    const Geom& g = p->geo;
    const Tiles& tl = p->tiles;
    const int T = 256;
    cudaMemsetAsync(p->d_cnt, 0, (tl.ntiles + 1) * sizeof(int), st);
    if (g.D == 2) k_ext<2, false><<<nblk(g.M, T), T, 0, st>>>(p->d_k0, g, tl, p->d_cnt, nullptr, nullptr);
    else k_ext<3, false><<<nblk(g.M, T), T, 0, st>>>(p->d_k0, g, tl, p->d_cnt, nullptr, nullptr);
    k_max_count<<<64, 256, 0, st>>>(p->d_cnt, tl.ntiles, p->d_flag + KP_FLAG_MAX_EXT);
    k_scan_excl<<<1, 1024, 0, st>>>(p->d_cnt, p->d_ext_off, tl.ntiles);
    cudaMemsetAsync(p->d_cnt, 0, (tl.ntiles + 1) * sizeof(int), st);
    if (g.D == 2) k_ext<2, true><<<nblk(g.M, T), T, 0, st>>>(p->d_k0, g, tl, p->d_cnt, p->d_ext_off, p->d_ext);
    else k_ext<3, true><<<nblk(g.M, T), T, 0, st>>>(p->d_k0, g, tl, p->d_cnt, p->d_ext_off, p->d_ext);
    p->launches += 5;
}

// The lists and items of the single-pass spreading variants for the current trajectory (when a
// plan tuned to a two-phase variant has to fall back to them).
kp_status build_spread_lists(kp_plan p, cudaStream_t st) {
    spread_lists_enqueue(p, st);
    KP_LAUNCH_CHECK();
    KP_TRY(build_spread_items(p, p->spread_chunk, st));
    p->lists_version = p->traj_version;
    return KP_OK;
}

kp_status set_trajectory_internal(kp_plan p, const float* traj, float traj_scale, cudaStream_t st) {
    if (!p || !traj) { set_error("null argument"); return KP_EINVAL; }
    const Geom& g = p->geo;
    const Tiles& tl = p->tiles;
    const int T = 256;
    drop_graphs(p);
    p->traj_set = false;
    p->traj_version++;
    p->circ_ok = false;
    if (traj != p->d_f)
        KP_TRY_CUDA(cudaMemcpyAsync(p->d_f, traj, (size_t)g.D * g.M * sizeof(float), cudaMemcpyDeviceToDevice, st));
    KP_TRY_CUDA(cudaMemsetAsync(p->d_ccnt, 0, (p->ncells + 1) * sizeof(int), st));
    KP_TRY_CUDA(cudaMemsetAsync(p->d_flag, 0, KP_NFLAGS * sizeof(int), st));
    if (g.D == 2) k_traj_key<2><<<nblk(g.M, T), T, 0, st>>>(traj, traj_scale, g, tl, p->cells_per_tile, p->d_key, p->d_ccnt, p->d_flag);
    else k_traj_key<3><<<nblk(g.M, T), T, 0, st>>>(traj, traj_scale, g, tl, p->cells_per_tile, p->d_key, p->d_ccnt, p->d_flag);
    KP_LAUNCH_CHECK();
    {
        // cell offsets by a multi-block exclusive scan, then the tile ranges and counts
        const unsigned nbk = (unsigned)((p->ncells + SCAN_B - 1) / SCAN_B);
        k_scan_part<<<nbk, SCAN_T, 0, st>>>(p->d_ccnt, p->ncells, p->d_scan_part);
        k_scan_excl<<<1, 1024, 0, st>>>(p->d_scan_part, p->d_scan_poff, nbk);
        k_scan_fin<<<nbk, SCAN_T, 0, st>>>(p->d_ccnt, p->ncells, p->d_scan_poff, p->d_coff);
        k_tile_off<<<nblk(tl.ntiles + 1, 256), 256, 0, st>>>(p->d_coff, tl.ntiles, p->cells_per_tile, p->d_off, p->d_cnt);
        KP_LAUNCH_CHECK();
        p->launches += 4;
    }
    k_max_count<<<64, 256, 0, st>>>(p->d_cnt, tl.ntiles, p->d_flag + 1);
    KP_LAUNCH_CHECK();
    KP_TRY_CUDA(cudaMemsetAsync(p->d_ccnt, 0, (p->ncells + 1) * sizeof(int), st));
    if (g.D == 2) k_traj_scatter<2><<<nblk(g.M, T), T, 0, st>>>(traj, traj_scale, g, p->d_key, p->d_coff, p->d_ccnt, p->d_perm, p->d_t, p->d_k0);
    else k_traj_scatter<3><<<nblk(g.M, T), T, 0, st>>>(traj, traj_scale, g, p->d_key, p->d_coff, p->d_ccnt, p->d_perm, p->d_t, p->d_k0);
    KP_LAUNCH_CHECK();
    KP_TRY(build_tap_tables(p, st));
    // per-tile spreading lists and items, used by the single-pass variants only: once the plan's
    // spreading is tuned to a two-phase variant (10-12) they are not built
    const bool lists = !(p->spread_tuned && p->spread_variant >= 10);
    if (lists) {
        spread_lists_enqueue(p, st);
        spread_items_counts(p, p->spread_chunk, st);
    }
    const unsigned tb = nblk(tl.ntiles, 256);
    k_ichunks<<<tb, 256, 0, st>>>(p->d_off, tl.ntiles, p->chunk, p->d_cnt);
    k_scan_excl<<<1, 1024, 0, st>>>(p->d_cnt, p->d_iitem_off, tl.ntiles);
    KP_LAUNCH_CHECK();
    own_items_counts(p, st);
    KP_LAUNCH_CHECK();
    p->launches += 11;
    if (!p->d_tslot) { set_error("plan without slot table"); return KP_EINTERNAL; }
    int cnt[8];
    KP_TRY(read_counts(p, p->d_iitem_off + tl.ntiles, p->d_tslot + tl.ntiles, cnt, st));
    if (cnt[0] != 0) {
        set_error(std::to_string(cnt[0]) + " trajectory coordinates outside [-N/2, N/2] or not finite");
        p->traj_set = false;
        return KP_EINVAL;
    }
    p->max_tile = lists ? cnt[2] : cnt[1];
    if (lists) {
        KP_TRY(spread_items_finish(p, p->spread_chunk, cnt[4], cnt[5], st));
        p->lists_version = p->traj_version;
    } else {
        p->n_split = 0;
    }
    // interpolation items (own samples of each tile, pieces of at most chunk)
    p->n_iitems = cnt[6];
    if (p->n_iitems > p->iitems_cap) {
        if (p->d_iitems) cudaFree(p->d_iitems);
        p->d_iitems = nullptr;
        KP_TRY_CUDA(cudaMalloc(&p->d_iitems, p->n_iitems * sizeof(int4)));
        p->iitems_cap = p->n_iitems;
    }
    k_iitems<<<tb, 256, 0, st>>>(p->d_off, p->d_iitem_off, tl.ntiles, p->chunk, p->d_iitems);
    KP_LAUNCH_CHECK();
    p->launches += 1;
    KP_TRY(sort_items_longest_first(p, p->d_iitems, p->n_iitems, p->chunk, st));
    KP_TRY(own_items_finish(p, cnt[7], st));
    p->traj_set = true;
    return autotune_spread(p, st);
}

}  // namespace kp

namespace kp {
kp_status report_timeout(kp_plan p, cudaStream_t st, const char* what) {
    KP_TRY_CUDA(cudaMemsetAsync(p->d_flag + KP_FLAG_TIMEOUT, 0, sizeof(int), st));
    KP_TRY_CUDA(cudaStreamSynchronize(st));
    set_error(what);
    return KP_ETIMEOUT;
}
}  // namespace kp

using namespace kp;

extern "C" {

const char* kp_status_string(kp_status s) {
    switch (s) {
        case KP_OK: return "KP_OK";
        case KP_EINVAL: return "KP_EINVAL";
        case KP_ENOMEM: return "KP_ENOMEM";
        case KP_ECUDA: return "KP_ECUDA";
        case KP_ECUFFT: return "KP_ECUFFT";
        case KP_EDIVERGED: return "KP_EDIVERGED";
        case KP_ENONFINITE: return "KP_ENONFINITE";
        case KP_ETIMEOUT: return "KP_ETIMEOUT";
        case KP_EINTERNAL: return "KP_EINTERNAL";
    }
    return "KP_UNKNOWN";
}

const char* kp_last_error(void) { return g_last_error.c_str(); }

kp_status kp_plan_create(kp_plan* out, const kp_params* params, void* stream) {
    KP_RANGE("kp_plan_create");
    g_last_error.clear();
    return plan_create_internal(out, params, false, (cudaStream_t)stream);
}

kp_status kp_plan_destroy(kp_plan plan) { return plan_destroy_internal(plan); }

kp_status kp_plan_set_trajectory(kp_plan plan, const float* traj_dev, void* stream) {
    KP_RANGE("kp_plan_set_trajectory");
    g_last_error.clear();
    if (!plan) { set_error("null plan"); return KP_EINVAL; }
    return set_trajectory_internal(plan, traj_dev, 1.0f, (cudaStream_t)stream);
}

kp_status kp_plan_set_maps(kp_plan plan, const void* maps_dev, kp_cdtype maps_t, void* stream) {
    KP_RANGE("kp_plan_set_maps");
    g_last_error.clear();
    if (!plan || !maps_dev) { set_error("null argument"); return KP_EINVAL; }
    if (plan->unit_maps) { set_error("plan has unit maps"); return KP_EINVAL; }
    if (maps_t != KP_C64 && maps_t != KP_C32_BF16 && maps_t != KP_C32_FP16) { set_error("bad maps type"); return KP_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = (int64_t)plan->geo.C * plan->geo.N;
    if (maps_t == KP_C64) k_copy_maps<float2><<<nblk(n, 256), 256, 0, st>>>((const float2*)maps_dev, (float2*)plan->d_maps, n);
    else k_copy_maps<unsigned><<<nblk(n, 256), 256, 0, st>>>((const unsigned*)maps_dev, (unsigned*)plan->d_maps, n);
    KP_LAUNCH_CHECK();
    plan->launches += 1;
    plan->maps_t = maps_t;
    plan->maps_set = true;
    plan->circ_ok = false;
    // cached graphs bake the maps type in: drop them
    drop_graphs(plan);
    return KP_OK;
}

kp_status kp_plan_launch_count(kp_plan plan, int64_t* count) {
    if (!plan || !count) { set_error("null argument"); return KP_EINVAL; }
    *count = plan->launches + (plan->pre_nufft ? plan->pre_nufft->launches : 0);
    return KP_OK;
}

kp_status kp_plan_set_wait_limit(kp_plan plan, long long cycles) {
    if (!plan) { set_error("null plan"); return KP_EINVAL; }
    if (cycles < 0) { set_error("the wait limit must be >= 0"); return KP_EINVAL; }
    plan->wait_cycles = cycles;
    drop_graphs(plan);
    return KP_OK;
}

kp_status kp_bounds_report(int* checked, uint32_t* count, uint32_t* first_site, int64_t* first_index) {
    uint32_t n = 0;
    unsigned long long first = 0;
#ifdef KP_CHECKED
    KP_TRY_CUDA(cudaDeviceSynchronize());
    for (auto take : oob_readers()) {
        unsigned int c = 0;
        unsigned long long f = 0;
        KP_TRY_CUDA(take(&c, &f));
        if (c && !n) first = f;
        n += c;
    }
    if (checked) *checked = 1;
#else
    if (checked) *checked = 0;
#endif
    if (count) *count = n;
    if (first_site) *first_site = n ? (uint32_t)(first >> 48) : 0u;
    if (first_index) *first_index = n ? (int64_t)(first & 0xFFFFFFFFFFFFull) : 0;
    return KP_OK;
}

kp_status kp_plan_sync(kp_plan plan, void* stream) {
    if (!plan) { set_error("null plan"); return KP_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    int timeout = 0;
    KP_TRY_CUDA(cudaMemcpyAsync(&timeout, plan->d_flag + KP_FLAG_TIMEOUT, sizeof(int), cudaMemcpyDeviceToHost, st));
    KP_TRY_CUDA(cudaStreamSynchronize(st));
    if (timeout) return report_timeout(plan, st, "a bounded device wait (bulk-copy staging of the interpolation) gave up");
    return KP_OK;
}

kp_status kp_plan_set_profiling(kp_plan plan, int enable) {
    if (!plan) { set_error("null plan"); return KP_EINVAL; }
    plan->profiling = enable != 0;
    return KP_OK;
}

kp_status kp_plan_spread_config(kp_plan plan, int* variant, int* chunk, int64_t* n_items, int64_t* n_split) {
    if (!plan) { set_error("null plan"); return KP_EINVAL; }
    if (!plan->traj_set) { set_error("no trajectory set"); return KP_EINVAL; }
    if (variant) *variant = plan->spread_variant;
    if (chunk) *chunk = plan->spread_chunk;
    if (n_items) *n_items = plan->n_items;
    if (n_split) *n_split = plan->n_split;
    return KP_OK;
}

kp_status kp_plan_tile_stats(kp_plan plan, int64_t* ntiles, int64_t* max_tile_samples) {
    if (!plan) { set_error("null plan"); return KP_EINVAL; }
    if (ntiles) *ntiles = plan->tiles.ntiles;
    if (max_tile_samples) *max_tile_samples = plan->max_tile;
    return KP_OK;
}

}  // extern "C"
