// Own 3D FFT of a plan's oversampled grids (all coils at once), used in place of cuFFT for 3D
// plans whose grid sizes factor into 2, 3 and 5 (Sec. 6's oversampled FFT, unnormalised in
// both directions like cuFFT: forward e^{-2 pi i n k / g}, inverse e^{+2 pi i n k / g}).
//
// One pass per axis.  A CTA takes 16 lines of one axis (8 for axes longer than 256 points): rows
// along x, or columns along y or z for 16 (8) consecutive x, so every global access is a 128-
// (64-) byte row segment.  The transform is a self-sorting (Stockham) mixed-radix one (radix 16,
// 8, 4, 2, 3 and 5 stages, and 10 and 15 where the odd part of the length fits one stage;
// 16, 8, 10 and 15 done as 4 x 4, 4 x 2, 2 x 5 and 3 x 5 in registers; twiddles from a table of
// the g-th roots of unity built on the host in float64).  Its first stage runs on the
// values each thread loads (all of its loads issued before any is used) and its last stage
// stores to global memory, so only the stages between them pass through shared memory, in
// place in one buffer of the CTA's lines.
//
// The passes exploit the structure of the NUFFT's grids.  The image occupies n_d of the g_d
// indices per axis (the band [0, n - n/2) and [g - n/2, g), where the pre-step puts it), and
// the adjoint reads only that crop back:
// * forward (x, then y, then z): the x pass transforms only the rows whose (z, y) lie in the
//   band and reads only their band points; the y pass takes only the z planes of the band and
//   reads only band rows; the z pass reads only band planes.  Points outside the band are zeros
//   that are never read.
// * inverse (z, then y, then x): the z pass writes only the band planes, the y pass transforms
//   only band planes and writes only band rows, the x pass only band rows and writes only band
//   points.  Afterwards only the crop holds the transform (the only part the adjoint reads).
#include "kp_internal.cuh"

#include <cmath>
#include <cstdlib>
#include <vector>

namespace kp {

constexpr int FF_LINES = 16;     // lines per CTA (at most)
// lines per CTA for length N: 16 up to 256 points (16 x = 128-byte row segments), else 8 so
// that the buffer of lines stays near 32 KB and five CTAs share an SM
constexpr int ff_lines(int N) { return N <= 256 ? 16 : 8; }
constexpr int FF_T = 256;        // threads per CTA
constexpr int FF_MAXN = 512;     // longest axis handled
constexpr int FF_MAXST = 10;     // radix stages at most

struct FfConst {                 // float64 on the host, rounded once
    float s3, c51, s51, c52, s52;   // sqrt(3)/2, cos and sin of 2 pi/5 and of 4 pi/5
    float2 w16[10];                 // (cos, sin) of 2 pi j / 16, j = 0..9 (radix-16 and radix-8 twiddles)
};

struct FfAxis {
    int N;                       // transform length (grid points along the axis)
    int nst;                     // radix stages
    int r[FF_MAXST];             // radices in the order applied
    const float2* tw;            // e^{-2 pi i m / N}, m in [0, N)
};

struct Fft3Plan {
    FfAxis ax[3];
    float2* d_tw = nullptr;
    FfConst k;
};

// The image samples the first forward pass forms itself (coil multiply and apodisation, the
// NUFFT's pre-step fused into the FFT): x, the maps (null: unit maps) and 1/Phi per axis.
struct PreSrc {
    const float2* x;
    const void* maps;
    const float* apod;
};

__device__ __forceinline__ bool in_band(int i, int n, int g) { return i < n - n / 2 || i >= g - n / 2; }
// pixel index of grid index i (i in the band)
__device__ __forceinline__ int pix_index(int i, int n, int g) { return i < n - n / 2 ? i + n / 2 : i - g + n / 2; }
__device__ __forceinline__ int band_index(int bi, int n, int g) { return bi < n - n / 2 ? bi : bi + (g - n); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// a * (-i s) for the forward sign (s = +1) or a * (+i) for the inverse (s = -1): (s a.y, -s a.x)
__device__ __forceinline__ float2 cmul_mi(float2 a, float s) { return make_float2(s * a.y, -s * a.x); }

// a e^{-s 2 pi i j / 16} for cs = (cos, sin)(2 pi j / 16)
__device__ __forceinline__ float2 cmul_w(float2 a, float2 cs, float s) {
    const float wy = -s * cs.y;
    return make_float2(a.x * cs.x - a.y * wy, a.x * wy + a.y * cs.x);
}

template <int R>
__device__ __forceinline__ void small_dft(float2* v, float s, const FfConst& k);

// 4-point DFT of (a, b, c, d) in place, outputs in natural order
__device__ __forceinline__ void dft4(float2& a, float2& b, float2& c, float2& d, float s) {
    const float2 t0 = cadd(a, c), t1 = csub(a, c), t2 = cadd(b, d), t3 = cmul_mi(csub(b, d), s);
    a = cadd(t0, t2);
    c = csub(t0, t2);
    b = cadd(t1, t3);
    d = csub(t1, t3);
}

// One R-point DFT of v[0..R-1] in place, sign s = +1 forward (omega = e^{-2 pi i / R}), -1 inverse.
// R = 16 and 8 run as 4 x 4 and 4 x 2 in registers: with q = 4 q1 + q2 (resp. 2 q1 + q2) and
// k = k1 + 4 k2, X[k] = sum_q2 w_R^(q2 k1) w^(q2 k2) [sum_q1 v[.] w_4^(q1 k1)].
template <int R>
__device__ __forceinline__ void small_dft(float2* v, float s, const FfConst& k) {
    static_assert(R == 2 || R == 3 || R == 4 || R == 5 || R == 8 || R == 16, "basic radix");
    if (R == 16) {
        float2 y[4][4];
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) {
            float2 a = v[q2], b = v[4 + q2], c = v[8 + q2], d = v[12 + q2];
            dft4(a, b, c, d, s);
            y[q2][0] = a;
            y[q2][1] = b;
            y[q2][2] = c;
            y[q2][3] = d;
        }
#pragma unroll
        for (int q2 = 1; q2 < 4; ++q2)
#pragma unroll
            for (int k1 = 1; k1 < 4; ++k1) y[q2][k1] = cmul_w(y[q2][k1], k.w16[q2 * k1], s);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 a = y[0][k1], b = y[1][k1], c = y[2][k1], d = y[3][k1];
            dft4(a, b, c, d, s);
            v[k1] = a;
            v[k1 + 4] = b;
            v[k1 + 8] = c;
            v[k1 + 12] = d;
        }
    } else if (R == 8) {
        float2 y0[4], y1[4];
        {
            float2 a = v[0], b = v[2], c = v[4], d = v[6];
            dft4(a, b, c, d, s);
            y0[0] = a; y0[1] = b; y0[2] = c; y0[3] = d;
        }
        {
            float2 a = v[1], b = v[3], c = v[5], d = v[7];
            dft4(a, b, c, d, s);
            y1[0] = a; y1[1] = b; y1[2] = c; y1[3] = d;
        }
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) y1[k1] = cmul_w(y1[k1], k.w16[2 * k1], s);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            v[k1] = cadd(y0[k1], y1[k1]);
            v[k1 + 4] = csub(y0[k1], y1[k1]);
        }
    } else if (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (R == 4) {
        const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        const float2 t2 = cadd(v[1], v[3]), t3 = cmul_mi(csub(v[1], v[3]), s);
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    } else if (R == 3) {
        // y1,2 = a0 - (a1 + a2)/2 -/+ i s sqrt(3)/2 (a1 - a2)
        const float2 sm = cadd(v[1], v[2]), d = cmul_mi(csub(v[1], v[2]), s * k.s3);
        const float2 m = make_float2(v[0].x - 0.5f * sm.x, v[0].y - 0.5f * sm.y);
        v[0] = cadd(v[0], sm);
        v[1] = cadd(m, d);
        v[2] = csub(m, d);
    } else {
        // R == 5: t1 = a1 + a4, t2 = a2 + a3, t3 = a1 - a4, t4 = a2 - a3;
        // y1,4 = a0 + c1 t1 + c2 t2 -/+ i (s1 t3 + s2 t4), y2,3 = a0 + c2 t1 + c1 t2 -/+ i (s2 t3 - s1 t4)
        const float2 a0 = v[0];
        const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]), t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
        const float2 p1 = make_float2(a0.x + k.c51 * t1.x + k.c52 * t2.x, a0.y + k.c51 * t1.y + k.c52 * t2.y);
        const float2 p2 = make_float2(a0.x + k.c52 * t1.x + k.c51 * t2.x, a0.y + k.c52 * t1.y + k.c51 * t2.y);
        const float2 q1 = cmul_mi(make_float2(k.s51 * t3.x + k.s52 * t4.x, k.s51 * t3.y + k.s52 * t4.y), s);
        const float2 q2 = cmul_mi(make_float2(k.s52 * t3.x - k.s51 * t4.x, k.s52 * t3.y - k.s51 * t4.y), s);
        v[0] = make_float2(a0.x + t1.x + t2.x, a0.y + t1.y + t2.y);
        v[1] = cadd(p1, q1);
        v[4] = csub(p1, q1);
        v[2] = cadd(p2, q2);
        v[3] = csub(p2, q2);
    }
}

// Radices of N in the order applied, at compile time (-1: N is not handled).  The
// power-of-two part goes greedily in 16s, 8s, 4s and 2s, then the odd part in 3s and 5s.  Where
// the last stage would still give every thread of the CTA a butterfly, the odd part runs as one
// radix instead (15 or 25, or 3 or 5 joined to the last power-of-two radix), which saves a
// round trip through shared memory: 240 = 16 x 15, 160 = 16 x 10, 480 = 16 x 2 x 15.  (Merges
// that leave threads idle in the last stage measured slower: 200 = 8 x 25 against 8 x 5 x 5,
// and the 320, 384 and 400 passes likewise.)  Radices 10, 15, 20, 24 and 25 are DFTs of two
// factors in registers (cdft).
constexpr int rad_list(int N, int* out) {
    int p = 1, o = N;
    while (o % 2 == 0) { o /= 2; p *= 2; }
    int c = 0;
    for (int f : {16, 8, 4, 2})
        while (p % f == 0) { p /= f; out[c++] = f; }
    int last = 0;                                   // the merged plan's last radix, 0: none
    if (o == 15 || o == 25) last = o;
    else if ((o == 3 || o == 5) && c >= 2) last = out[c - 1] * o;
    if (last && ff_lines(N) * (N / last) >= FF_T) {
        if (last == o) out[c++] = o;
        else out[c - 1] = last;
        return c;
    }
    for (int f : {3, 5})
        while (o % f == 0) { o /= f; out[c++] = f; }
    return o == 1 ? c : -1;
}
constexpr int rad_count(int N) {
    int r[16] = {};
    return rad_list(N, r);
}
constexpr int rad_at(int N, int i) {
    int r[16] = {};
    const int c = rad_list(N, r);
    return i < c ? r[i] : 1;
}

// Factors (P, Q) of a radix done as a two-factor DFT; P = 0 for the basic radices.
constexpr int split_p(int R) { return R == 10 ? 2 : R == 15 ? 3 : R == 20 ? 4 : R == 24 ? 8 : R == 25 ? 5 : 0; }

// R-point DFT of v in place for a radix of length-N passes.  A radix R = P Q of split_p runs as
// Cooley-Tukey in registers: with q = Q q1 + q2 and k = k1 + P k2, X[k] = sum_q2 w_R^(q2 k1)
// w_Q^(q2 k2) [sum_q1 v[q] w_P^(q1 k1)]; the w_R twiddles are the table's w_N^(q2 k1 N / R).
template <int R, int N>
__device__ __forceinline__ void cdft(float2* v, float s, const FfConst& k, const float2* tw) {
    constexpr int P = split_p(R);
    if constexpr (P == 0) {
        small_dft<R>(v, s, k);
    } else {
        constexpr int Q = R / P;
        static_assert(P * Q == R && N % R == 0, "radix splits and divides the length");
        float2 y[Q][P];
#pragma unroll
        for (int q2 = 0; q2 < Q; ++q2) {
#pragma unroll
            for (int q1 = 0; q1 < P; ++q1) y[q2][q1] = v[Q * q1 + q2];
            small_dft<P>(y[q2], s, k);
        }
#pragma unroll
        for (int q2 = 1; q2 < Q; ++q2)
#pragma unroll
            for (int k1 = 1; k1 < P; ++k1) {
                float2 w = tw[q2 * k1 * (N / R)];
                w.y *= s;
                const float2 a = y[q2][k1];
                y[q2][k1] = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
            }
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
            float2 b[Q];
#pragma unroll
            for (int q2 = 0; q2 < Q; ++q2) b[q2] = y[q2][k1];
            small_dft<Q>(b, s, k);
#pragma unroll
            for (int k2 = 0; k2 < Q; ++k2) v[k1 + P * k2] = b[k2];
        }
    }
}

// Shared-memory position of element n of line l: l * N + n when XL (rows along x), else
// n * LN + l (LN lines side by side, as they lie in global memory).
template <int N, bool XL>
__device__ __forceinline__ int sidx(int l, int n) { return XL ? l * N + n : n * ff_lines(N) + l; }

// a * w for the twiddle w = tw[e] = e^{-2 pi i e / N}, conjugated for the inverse (s = -1)
__device__ __forceinline__ float2 twiddle(float2 x, float2 w, float s) {
    w.y *= s;
    return make_float2(x.x * w.x - x.y * w.y, x.x * w.y + x.y * w.x);
}

// Stockham, decimation in time: stage ST (radix r) combines r transforms of length L into one
// of length L r; butterfly (j, kk) (j < m = N / (L r), kk < L) takes elements kk N / L + j + q m,
// q < r, multiplies input q by w^(q kk m) (w = e^{-+2 pi i / N}) and puts output t of its r-point
// DFT at (kk + L t) m + j.  The first stage (L = 1, no twiddles) runs on the values loaded from
// global memory and the last one (m = 1) stores to global memory, so only the stages between
// them go through shared memory: here, in place in `a`, every thread reading all its
// butterflies' inputs (and transforming them) before the CTA's barrier, then writing.
template <int N, bool XL, int ST, int L>
__device__ __forceinline__ void stockham_mid(float2* a, const float2* tw, float s, const FfConst& k) {
    constexpr int LN = ff_lines(N);
    if constexpr (ST + 1 >= rad_count(N)) {
        return;
    } else {
        constexpr int r = rad_at(N, ST), Lr = L * r, m = N / Lr, nb = N / r, NL = N / L;
        constexpr int NB = LN * nb, BPT = (NB + FF_T - 1) / FF_T;
        float2 v[BPT][r];
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const int it = threadIdx.x + b * FF_T;
            if (it < NB) {
                const int l = XL ? it / nb : it % LN;
                const int bf = XL ? it - l * nb : it / LN;
                const int j = bf % m, kk = bf / m;
#pragma unroll
                for (int q = 0; q < r; ++q) {
                    const float2 x = a[sidx<N, XL>(l, kk * NL + j + q * m)];
                    v[b][q] = q > 0 ? twiddle(x, tw[q * kk * m], s) : x;
                }
                cdft<r, N>(v[b], s, k, tw);
            }
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const int it = threadIdx.x + b * FF_T;
            if (it < NB) {
                const int l = XL ? it / nb : it % LN;
                const int bf = XL ? it - l * nb : it / LN;
                const int j = bf % m, kk = bf / m;
#pragma unroll
                for (int t = 0; t < r; ++t) a[sidx<N, XL>(l, (kk + L * t) * m + j)] = v[b][t];
            }
        }
        __syncthreads();
        stockham_mid<N, XL, ST + 1, Lr>(a, tw, s, k);
    }
}

// Pass along AXIS (0 = z, 1 = y, 2 = x) of every coil's grid; INV selects the inverse.  Line
// selection and pruning as in the file header.
template <int AXIS, bool INV, int N, bool PRE = false, typename MT = float2>
__global__ void __launch_bounds__(FF_T) k_fft_pass(const float2* in, float2* out, Geom geo, FfAxis ax, FfConst k,
                                                   PreSrc pre) {
    // (no __restrict__: the y, z and inverse passes work in place, each CTA on its own lines, all
    // of whose loads are issued in the first stage, before the barrier that precedes any store)
    // PRE (first forward pass only): the band points are s_c x / Phi, formed from `pre`, not read
    constexpr int LN = ff_lines(N), NST = rad_count(N);
    static_assert(NST >= 2, "the first and last stages are distinct");
    constexpr bool XL = AXIS == 2;
    extern __shared__ __align__(16) float2 fsm[];
    float2* A = fsm;                                    // [LN lines][N]
    float2* tw = A + LN * N;
    for (int i = threadIdx.x; i < N; i += FF_T) tw[i] = ax.tw[i];
    const int g0 = geo.g[0], g1 = geo.g[1], g2 = geo.g[2];
    const int n0 = geo.n[0], n1 = geo.n[1], n2 = geo.n[2];
    const bool load_band = !INV, store_band = INV;      // forward reads only the band, inverse writes only it
    // per line: base offset of element 0, or -1 when the line does not exist; element n at base + n stride
    __shared__ int64_t base_s[FF_LINES];
    __shared__ int64_t pix_s[FF_LINES];                 // PRE: maps offset of the row's first pixel
    __shared__ int64_t img_s[FF_LINES];                 // PRE: image offset of the row's first pixel
    __shared__ float apod_s[FF_LINES];                  // PRE: 1/Phi of the row's z and y
    int64_t stride;
    if (AXIS == 2) {
        stride = 1;
        if (threadIdx.x < LN) {
            const int64_t row = (int64_t)blockIdx.x * LN + threadIdx.x;
            const int64_t nrows = (int64_t)geo.C * n0 * n1;
            if (row < nrows) {
                // coil fastest: a CTA's rows are few image rows in every coil, so the fused
                // pre-step's image and 1/Phi loads of a row are shared by its coils
                const int c = (int)(row % geo.C);
                const int rem = (int)(row / geo.C);
                const int z = band_index(rem / n1, n0, g0), y = band_index(rem % n1, n1, g1);
                base_s[threadIdx.x] = (int64_t)c * geo.G + ((int64_t)z * g1 + y) * g2;
                if (PRE) {
                    const int pz = pix_index(z, n0, g0), py = pix_index(y, n1, g1);
                    img_s[threadIdx.x] = ((int64_t)pz * n1 + py) * n2;
                    pix_s[threadIdx.x] = (int64_t)c * geo.N + img_s[threadIdx.x];
                    apod_s[threadIdx.x] = pre.apod[pz] * pre.apod[n0 + py];
                }
            } else {
                base_s[threadIdx.x] = -1;
            }
        }
    } else {
        // CTA: one (coil, outer index, x block); AXIS 1: outer = band plane z; AXIS 0: outer = row y
        const int xblocks = (g2 + LN - 1) / LN;
        const int outer_n = AXIS == 1 ? n0 : g1;
        const int xb = blockIdx.x % xblocks;
        const int rest = blockIdx.x / xblocks;
        const int o = rest % outer_n, c = rest / outer_n;
        stride = AXIS == 1 ? (int64_t)g2 : (int64_t)g1 * g2;
        if (threadIdx.x < LN) {
            const int x = xb * LN + threadIdx.x;
            if (x < g2) {
                const int64_t ob = AXIS == 1 ? (int64_t)band_index(o, n0, g0) * g1 * g2 : (int64_t)o * g2;
                base_s[threadIdx.x] = (int64_t)c * geo.G + ob + x;
            } else {
                base_s[threadIdx.x] = -1;
            }
        }
    }
    __syncthreads();
    const int nb_axis = AXIS == 0 ? n0 : (AXIS == 1 ? n1 : n2);
    const float s = INV ? -1.f : 1.f;
    // first stage (radix r0, L = 1) on the loaded values: every load of this thread is issued
    // before any is used (zeros for missing lines and, in the forward direction, outside the
    // band); butterfly j of line l takes elements j + q m0 (consecutive threads: consecutive j
    // of a row, or consecutive lines, so each load instruction reads whole row segments)
    {
        constexpr int r0 = rad_at(N, 0), m0 = N / r0, NB = LN * m0, BPT = (NB + FF_T - 1) / FF_T;
        float2 v[BPT][r0];
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const int it = threadIdx.x + b * FF_T;
            const int l = XL ? it / m0 : it % LN;
            const int j = XL ? it - l * m0 : it / LN;
            const int64_t bs = it < NB ? base_s[l] : -1;
#pragma unroll
            for (int q = 0; q < r0; ++q) {
                const int n = j + q * m0;
                v[b][q] = make_float2(0.f, 0.f);
                if (bs >= 0 && (!load_band || in_band(n, nb_axis, N))) {
                    if constexpr (PRE) {
                        // the pre-step's arithmetic, in its order: x (1/Phi_z 1/Phi_y 1/Phi_x), then s_c times it
                        const int px = pix_index(n, n2, g2);
                        if (KP_INB(3, px, n2) && KP_INB(3, img_s[l] + px, geo.N) &&
                            (!pre.maps || KP_INB(3, pix_s[l] + px, (int64_t)geo.C * geo.N))) {
                            const float a = apod_s[l] * pre.apod[n0 + n1 + px];
                            float2 xv = pre.x[img_s[l] + px];
                            xv.x *= a;
                            xv.y *= a;
                            const float2 sv = pre.maps ? ldc<MT>((const MT*)pre.maps, pix_s[l] + px) : make_float2(1.f, 0.f);
                            v[b][q] = cmul(sv, xv);
                        }
                    } else if (KP_INB(1, bs + n * stride, (int64_t)geo.C * geo.G)) {
                        v[b][q] = in[bs + n * stride];
                    }
                }
            }
        }
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const int it = threadIdx.x + b * FF_T;
            if (it < NB) {
                const int l = XL ? it / m0 : it % LN;
                const int j = XL ? it - l * m0 : it / LN;
                cdft<r0, N>(v[b], s, k, tw);
#pragma unroll
                for (int t = 0; t < r0; ++t) A[sidx<N, XL>(l, t * m0 + j)] = v[b][t];
            }
        }
    }
    __syncthreads();
    stockham_mid<N, XL, 1, rad_at(N, 0)>(A, tw, s, k);
    // last stage (radix rl, m = 1): butterfly kk of line l takes elements kk rl + q and stores
    // output t at kk + L t, straight to global memory (the inverse only inside the band)
    {
        constexpr int rl = rad_at(N, NST - 1), L = N / rl, NB = LN * L, BPT = (NB + FF_T - 1) / FF_T;
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const int it = threadIdx.x + b * FF_T;
            if (it < NB) {
                const int l = XL ? it / L : it % LN;
                const int kk = XL ? it - l * L : it / LN;
                float2 v[rl];
#pragma unroll
                for (int q = 0; q < rl; ++q) {
                    const float2 x = A[sidx<N, XL>(l, kk * rl + q)];
                    v[q] = q > 0 ? twiddle(x, tw[q * kk], s) : x;
                }
                cdft<rl, N>(v, s, k, tw);
                const int64_t bs = base_s[l];
                if (bs >= 0) {
#pragma unroll
                    for (int t = 0; t < rl; ++t) {
                        const int n = kk + L * t;
                        if ((!store_band || in_band(n, nb_axis, N)) && KP_INB(2, bs + n * stride, (int64_t)geo.C * geo.G))
                            out[bs + n * stride] = v[t];
                    }
                }
            }
        }
    }
}

static size_t pass_smem(int N) { return ((size_t)(N <= 256 ? 16 : 8) * N + N) * sizeof(float2); }

// Radices of N as the passes apply them (rad_list); false if N is not handled.
static bool factor(int N, FfAxis& ax) {
    int r[16] = {};
    const int c = rad_list(N, r);
    if (c < 2 || c > FF_MAXST) return false;
    ax.nst = c;
    for (int i = 0; i < c; ++i) ax.r[i] = r[i];
    return true;
}

static bool size_compiled(int N);

// Passes and twiddle tables for grids of g[0] x g[1] x g[2] points; null when some length has no
// compiled passes (or KPDHG_FFT=cufft).
Fft3Plan* fft3_make(const int g[3]) {
    const char* env = std::getenv("KPDHG_FFT");
    if (env && std::string(env) == "cufft") return nullptr;       // cuFFT when asked for
    Fft3Plan f{};
    size_t tot = 0;
    for (int d = 0; d < 3; ++d) {
        FfAxis& ax = f.ax[d];
        ax.N = g[d];
        if (ax.N > FF_MAXN || !factor(ax.N, ax) || !size_compiled(ax.N)) return nullptr;
        tot += ax.N;
    }
    // twiddle tables e^{-2 pi i m / N} in float64, rounded once
    std::vector<float2> h(tot);
    size_t o = 0;
    for (int d = 0; d < 3; ++d) {
        const int N = f.ax[d].N;
        for (int m = 0; m < N; ++m) {
            const double a = -2.0 * M_PI * (double)m / (double)N;
            h[o + m] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
        o += N;
    }
    Fft3Plan* q = new (std::nothrow) Fft3Plan(f);
    if (!q) return nullptr;
    if (cudaMalloc(&q->d_tw, tot * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        delete q;
        return nullptr;
    }
    if (cudaMemcpy(q->d_tw, h.data(), tot * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(q->d_tw);
        delete q;
        return nullptr;
    }
    o = 0;
    for (int d = 0; d < 3; ++d) {
        q->ax[d].tw = q->d_tw + o;
        o += q->ax[d].N;
    }
    q->k.s3 = (float)(std::sqrt(3.0) / 2.0);
    q->k.c51 = (float)std::cos(2.0 * M_PI / 5.0);
    q->k.s51 = (float)std::sin(2.0 * M_PI / 5.0);
    q->k.c52 = (float)std::cos(4.0 * M_PI / 5.0);
    q->k.s52 = (float)std::sin(4.0 * M_PI / 5.0);
    for (int j = 0; j < 10; ++j)
        q->k.w16[j] = make_float2((float)std::cos(2.0 * M_PI * j / 16.0), (float)std::sin(2.0 * M_PI * j / 16.0));
    return q;
}

void fft3_free(Fft3Plan* f) {
    if (!f) return;
    if (f->d_tw) cudaFree(f->d_tw);
    delete f;
}

kp_status fft3_create(kp_plan p) {
    if (p->geo.D == 3) p->fft3 = fft3_make(p->geo.g);
    return KP_OK;
}

void fft3_destroy(kp_plan p) {
    fft3_free(p->fft3);
    p->fft3 = nullptr;
}

// Grid sizes with compiled passes (the 3D workloads' grids and their preconditioner's 2N grids,
// and small test grids); a plan with another size keeps cuFFT.
#define KP_FFT_SIZES(X) X(20) X(30) X(40) X(60) X(80) X(100) X(120) X(160) X(200) X(240) X(320) X(384) X(400) X(480)

static bool size_compiled(int N) {
    switch (N) {
#define KP_FFT_CASE(n) case n:
        KP_FFT_SIZES(KP_FFT_CASE)
#undef KP_FFT_CASE
        return true;
        default: return false;
    }
}

template <int AXIS, bool INV, int N, bool PRE = false, typename MT = float2>
static kp_status launch_pass_n(const Fft3Plan* f, const Geom& g, const float2* in, float2* out, unsigned nblocks,
                               const PreSrc& pre, cudaStream_t st) {
    static PerDeviceOnce attr;
    if (attr.first())
        KP_TRY_CUDA(cudaFuncSetAttribute(k_fft_pass<AXIS, INV, N, PRE, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pass_smem(N)));
    k_fft_pass<AXIS, INV, N, PRE, MT><<<nblocks, FF_T, pass_smem(N), st>>>(in, out, g, f->ax[AXIS], f->k, pre);
    KP_LAUNCH_CHECK();
    return KP_OK;
}

template <int AXIS, bool INV, bool PRE = false, typename MT = float2>
static kp_status launch_pass(const Fft3Plan* f, const Geom& g, int64_t& launches, const float2* in, float2* out,
                             cudaStream_t st, const PreSrc& pre = PreSrc{}) {
    int64_t nblocks;
    const int ln = g.g[AXIS] <= 256 ? 16 : 8;           // ff_lines(N) of this pass
    const int64_t xblocks = (g.g[2] + ln - 1) / ln;
    if (AXIS == 2) nblocks = ((int64_t)g.C * g.n[0] * g.n[1] + ln - 1) / ln;
    else if (AXIS == 1) nblocks = (int64_t)g.C * g.n[0] * xblocks;
    else nblocks = (int64_t)g.C * g.g[1] * xblocks;
    if (nblocks > INT32_MAX) { set_error("grid too large for the FFT passes"); return KP_EINVAL; }
    launches += 1;
    switch (g.g[AXIS]) {
#define KP_FFT_CASE(n) case n: return launch_pass_n<AXIS, INV, n, PRE, MT>(f, g, in, out, (unsigned)nblocks, pre, st);
        KP_FFT_SIZES(KP_FFT_CASE)
#undef KP_FFT_CASE
        default: set_error("FFT pass size without compiled kernel"); return KP_EINTERNAL;
    }
}

kp_status fft3_forward_geo(const Fft3Plan* f, const Geom& g, const float2* in, float2* out, int64_t& launches,
                           cudaStream_t st) {
    KP_TRY((launch_pass<2, false>(f, g, launches, in, out, st)));
    KP_TRY((launch_pass<1, false>(f, g, launches, out, out, st)));
    return launch_pass<0, false>(f, g, launches, out, out, st);
}

kp_status fft3_inverse_geo(const Fft3Plan* f, const Geom& g, float2* io, int64_t& launches, cudaStream_t st) {
    KP_TRY((launch_pass<0, true>(f, g, launches, io, io, st)));
    KP_TRY((launch_pass<1, true>(f, g, launches, io, io, st)));
    return launch_pass<2, true>(f, g, launches, io, io, st);
}

kp_status fft3_forward(kp_plan p, const float2* in, float2* out, cudaStream_t st) {
    return fft3_forward_geo(p->fft3, p->geo, in, out, p->launches, st);
}

kp_status fft3_forward_image(kp_plan p, const float2* x, cudaStream_t st) {
    const PreSrc pre{x, p->unit_maps ? nullptr : p->d_maps, p->d_apod};
    const Fft3Plan* f = p->fft3;
    const Geom& g = p->geo;
    float2* out = p->d_gridF;
    switch (p->unit_maps ? KP_C64 : p->maps_t) {
        case KP_C64: KP_TRY((launch_pass<2, false, true, float2>(f, g, p->launches, nullptr, out, st, pre))); break;
        case KP_C32_BF16: KP_TRY((launch_pass<2, false, true, __nv_bfloat162>(f, g, p->launches, nullptr, out, st, pre))); break;
        default: KP_TRY((launch_pass<2, false, true, __half2>(f, g, p->launches, nullptr, out, st, pre))); break;
    }
    KP_TRY((launch_pass<1, false>(f, g, p->launches, out, out, st)));
    return launch_pass<0, false>(f, g, p->launches, out, out, st);
}

kp_status fft3_inverse(kp_plan p, float2* io, cudaStream_t st) {
    return fft3_inverse_geo(p->fft3, p->geo, io, p->launches, st);
}

}  // namespace kp
