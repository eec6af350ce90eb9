// l2-optimised diagonal k-space preconditioner (Sec. 5, App. A), fast route of Sec. 5.1:
//
//   q_cd = s_c s_d^*  zero-padded to the 2N grid  -> FFT -> R_c = sum_d |Q_cd|^2
//   r_c  = IFFT(R_c) / (2^D N)                      (autocorrelation sum, lags in [-N_d, N_d))
//   h    = N^{-1/2} sum_j e^{+i 2 pi f_j k/N}        (type-1 NUFFT of ones at 2 f_j on the 2N image)
//   p_c[i] = ||s_c||^2 sqrt(N) / Re(sum_k r_c[k] h[k] e^{-i 2 pi f_i k / N})   (type-2 NUFFT at 2 f_i)
//
// FFTs and gridding run in float32; the denominator sums (R_c over coil pairs, and the
// interpolation taps of the last type-2 step, real part only) accumulate in float64.
// With the 2N-image NUFFT carrying (2^D N)^{-1/2} in both directions, the last line is
// p_c[i] = ||s_c||^2 / (2^D Re(fwd_2N(r_c * adj_2N(1))[i])).  Pairs (c, d) and (d, c) share
// one FFT: |Q_dc|^2[m] = |Q_cd|^2[-m].  Single channel (Eq. sc_precond): C = 1, s = 1.
#include "kp_internal.cuh"

#include <algorithm>
#include <vector>

namespace kp {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Device memory the construction may use for a batch of 2N-grid spectra: an eighth of the
// free memory when the plan's construction is first set up, between 256 MB and 20 GB (every
// pair spectrum of a 192^3 image with 8 coils, 36 x 453 MB, fits at once on a GB300).
static size_t pre_batch_bytes() {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        fr = 0;
    }
    return std::min<size_t>(std::max<size_t>(fr / 8, (size_t)256 << 20), (size_t)20 << 30);
}

struct PrePlan {
    int D = 0;
    int nb[MAXD] = {1, 1, 1};
    int64_t Nb = 0;
    int C = 0;            // coils of the owning plan
    int B = 0;            // pairs per FFT batch (all pairs when they fit in the budget below)
    int Cb = 0;           // coils per batch of the r_c -> v_c steps
    double* d_R = nullptr;      // [C][Nb]
    float2* d_q = nullptr;      // [B][Nb]
    float2* d_r = nullptr;      // [Cb][Nb]
    float2* d_h = nullptr;      // [Nb]
    float2* d_v = nullptr;      // [Cb][Nb]
    double* d_norm = nullptr;   // [C]
    int2* d_pairs = nullptr;    // [C(C+1)/2]
    int npairs = 0;
    cufftHandle fft_pairs = 0, fft_one = 0, fft_coils = 0;
    bool ok_pairs = false, ok_one = false, ok_coils = false;
    Fft3Plan* f3 = nullptr;     // own passes on the 2N grid (3D, compiled lengths), else the cuFFT plans
    int traj_version = -1;
};

void pre_destroy(kp_plan p) {
    if (p->pre_nufft) { plan_destroy_internal(p->pre_nufft); p->pre_nufft = nullptr; }
    PrePlan* q = p->pre;
    if (!q) return;
    if (q->ok_pairs) cufftDestroy(q->fft_pairs);
    if (q->ok_one) cufftDestroy(q->fft_one);
    if (q->ok_coils) cufftDestroy(q->fft_coils);
    fft3_free(q->f3);
    void* bufs[] = {q->d_R, q->d_q, q->d_r, q->d_h, q->d_v, q->d_norm, q->d_pairs};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete q;
    p->pre = nullptr;
}

// Geometry of `count` 2N grids for the own FFT passes: image band of the owning plan's image
// (the products' support), or the whole grid (full = true: no pruning).
static Geom pre_geo(const PrePlan* q, const Geom& g, int count, bool full) {
    Geom r{};
    r.D = 3;
    r.C = count;
    r.N = 1;
    for (int d = 0; d < 3; ++d) {
        r.g[d] = q->nb[d];
        r.n[d] = full ? q->nb[d] : g.n[d];
        r.N *= r.n[d];
    }
    r.G = q->Nb;
    return r;
}

static kp_status pre_create(kp_plan p, cudaStream_t st) {
    if (p->pre) return KP_OK;
    PrePlan* q = new (std::nothrow) PrePlan();
    if (!q) { set_error("host allocation failed"); return KP_ENOMEM; }
    p->pre = q;
    const Geom& g = p->geo;
    q->D = g.D;
    q->C = g.C;
    q->Nb = 1;
    for (int d = 0; d < g.D; ++d) { q->nb[d] = 2 * g.n[d]; q->Nb *= q->nb[d]; }
    if (q->Nb >= ((int64_t)1 << 31)) {
        // the construction indexes the 2N grid (and the 2N plan's oversampled grid) in 32 bits
        set_error("preconditioner: the 2N image has 2^31 points or more");
        return KP_EINVAL;
    }
    q->npairs = g.C * (g.C + 1) / 2;
    // every pair spectrum at once when they fit in PRE_BATCH_BYTES (one FFT batch, R written
    // once per coil), else batches of 16 (2D) or 2 (3D) accumulated into R
    const size_t grid_bytes = (size_t)q->Nb * sizeof(float2);
    const size_t budget = pre_batch_bytes();
    const int bmax = g.D == 2 ? 16 : 2;
    if ((size_t)q->npairs * grid_bytes <= budget) q->B = q->npairs;
    else q->B = q->npairs < bmax ? q->npairs : bmax;
    q->Cb = (int)std::max<size_t>(1, std::min<size_t>((size_t)g.C, budget / (2 * grid_bytes)));
    KP_TRY_CUDA(cudaMalloc(&q->d_R, (size_t)g.C * q->Nb * sizeof(double)));
    KP_TRY_CUDA(cudaMalloc(&q->d_q, (size_t)q->B * q->Nb * sizeof(float2)));
    KP_TRY_CUDA(cudaMalloc(&q->d_r, (size_t)q->Cb * q->Nb * sizeof(float2)));
    KP_TRY_CUDA(cudaMalloc(&q->d_h, (size_t)q->Nb * sizeof(float2)));
    KP_TRY_CUDA(cudaMalloc(&q->d_v, (size_t)q->Cb * q->Nb * sizeof(float2)));
    KP_TRY_CUDA(cudaMalloc(&q->d_norm, (size_t)g.C * sizeof(double)));
    std::vector<int2> pairs;
    for (int c = 0; c < g.C; ++c)
        for (int d = c; d < g.C; ++d) pairs.push_back(make_int2(c, d));
    KP_TRY_CUDA(cudaMalloc(&q->d_pairs, pairs.size() * sizeof(int2)));
    KP_TRY_CUDA(cudaMemcpy(q->d_pairs, pairs.data(), pairs.size() * sizeof(int2), cudaMemcpyHostToDevice));
    int dims[3] = {q->nb[0], q->nb[1], q->nb[2]};
    if (cufftPlanMany(&q->fft_pairs, g.D, dims, nullptr, 1, (int)q->Nb, nullptr, 1, (int)q->Nb, CUFFT_C2C, q->B) !=
        CUFFT_SUCCESS) {
        // no room for the whole batch's work area: batches of bmax pairs accumulated into R
        cudaGetLastError();
        const int b2 = q->npairs < bmax ? q->npairs : bmax;
        if (b2 >= q->B) { set_error("cuFFT plan of the pair spectra failed"); return KP_ECUFFT; }
        q->B = b2;
        cudaFree(q->d_q);
        q->d_q = nullptr;
        KP_TRY_CUDA(cudaMalloc(&q->d_q, (size_t)q->B * q->Nb * sizeof(float2)));
        KP_TRY_CUFFT(cufftPlanMany(&q->fft_pairs, g.D, dims, nullptr, 1, (int)q->Nb, nullptr, 1, (int)q->Nb, CUFFT_C2C, q->B));
    }
    q->ok_pairs = true;
    KP_TRY_CUFFT(cufftPlanMany(&q->fft_one, g.D, dims, nullptr, 1, (int)q->Nb, nullptr, 1, (int)q->Nb, CUFFT_C2C, 1));
    q->ok_one = true;
    KP_TRY_CUFFT(cufftPlanMany(&q->fft_coils, g.D, dims, nullptr, 1, (int)q->Nb, nullptr, 1, (int)q->Nb, CUFFT_C2C, q->Cb));
    q->ok_coils = true;
    if (g.D == 3) q->f3 = fft3_make(q->nb);
    // NUFFT on the 2N image with unit maps and one coil
    kp_params prm = p->P;
    prm.ncoils = 1;
    prm.wavelet_levels = 0;
    for (int d = 0; d < g.D; ++d) prm.img[d] = 2 * g.n[d];
    KP_TRY(plan_create_internal(&p->pre_nufft, &prm, true, st));
    if (p->pre_nufft->geo.G >= ((int64_t)1 << 31)) {
        set_error("preconditioner: the 2N image's oversampled grid has 2^31 points or more");
        return KP_EINVAL;
    }
    return KP_OK;
}

// Zero-padded product q = s_c s_d^* (or 1 with unit maps) on the 2N grid, pixel n at n mod 2N.
template <typename MT>
__global__ void k_make_q(const MT* __restrict__ maps, const int2* __restrict__ pairs, int pair0, int npairs_valid,
                         Geom geo, int D, int nb0, int nb1, int nb2, int64_t Nb, int B, float2* __restrict__ q) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Nb) return;
    const int nb[3] = {nb0, nb1, nb2};
    int ii[MAXD];
    int64_t r = m;
    for (int d = D - 1; d >= 0; --d) { ii[d] = (int)(r % nb[d]); r /= nb[d]; }
    int64_t j = 0;
    bool inside = true;
    for (int d = 0; d < D; ++d) {
        int n = geo.n[d], h = n / 2;
        int jd = ii[d] < n - h ? ii[d] + h : (ii[d] >= nb[d] - h ? ii[d] - nb[d] + h : -1);
        if (jd < 0) inside = false;
        j = j * n + (jd < 0 ? 0 : jd);
    }
    for (int b = 0; b < B; ++b) {
        float2 v = make_float2(0.f, 0.f);
        if (inside && b < npairs_valid) {
            if (maps) {
                int2 cd = pairs[pair0 + b];
                float2 sc = ldc<MT>(maps, (size_t)cd.x * geo.N + j);
                float2 sd = ldc<MT>(maps, (size_t)cd.y * geo.N + j);
                v = cmulc(sd, sc);   // s_c s_d^*
            } else {
                v = make_float2(1.f, 0.f);
            }
        }
        q[(size_t)b * Nb + m] = v;
    }
}

// R_c[m] += |Q_cd[m]|^2, R_d[m] += |Q_cd[-m]|^2 for each pair of the batch (float64).
__global__ void k_accum_R(const float2* __restrict__ Q, const int2* __restrict__ pairs, int pair0, int npairs_valid,
                          int D, int nb0, int nb1, int nb2, int64_t Nb, double* __restrict__ R, bool unit) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Nb) return;
    const int nb[3] = {nb0, nb1, nb2};
    // index of -m
    int64_t r = m, mneg = 0, stride = 1;
    for (int d = D - 1; d >= 0; --d) {
        int i = (int)(r % nb[d]);
        r /= nb[d];
        int in = i == 0 ? 0 : nb[d] - i;
        mneg += in * stride;
        stride *= nb[d];
    }
    for (int b = 0; b < npairs_valid; ++b) {
        int2 cd = unit ? make_int2(0, 0) : pairs[pair0 + b];
        float2 a = Q[(size_t)b * Nb + m];
        R[(size_t)cd.x * Nb + m] += (double)a.x * a.x + (double)a.y * a.y;
        if (cd.y != cd.x) {
            float2 bq = Q[(size_t)b * Nb + mneg];
            R[(size_t)cd.y * Nb + m] += (double)bq.x * bq.x + (double)bq.y * bq.y;
        }
    }
}

// Index of the frequency -m (periodic) on the 2N grid, m < 2^31.
__device__ __forceinline__ unsigned neg_index(unsigned m, int D, unsigned nb0, unsigned nb1, unsigned nb2) {
    if (D == 2) {
        const unsigned i1 = m % nb1, i0 = m / nb1;
        return (i0 ? nb0 - i0 : 0u) * nb1 + (i1 ? nb1 - i1 : 0u);
    }
    const unsigned i2 = m % nb2, r = m / nb2, i1 = r % nb1, i0 = r / nb1;
    return ((i0 ? nb0 - i0 : 0u) * nb1 + (i1 ? nb1 - i1 : 0u)) * nb2 + (i2 ? nb2 - i2 : 0u);
}

// |q|^2 as a float-float value (both squares exact, one rounding in the sum's low part)
__device__ __forceinline__ ff32 ff_abs2(float2 q) { return ff_add(ff_two_prod(q.x, q.x), ff_two_prod(q.y, q.y)); }

// With every pair's spectrum in Q (pair (c, d), c <= d, at index c C - c (c - 1) / 2 + d - c):
// R_c[m] = sum_{d >= c} |Q_cd[m]|^2 + sum_{d < c} |Q_dc[-m]|^2, summed in float-float (about 48
// bits: the float64 pipe would bound this pass) and written once as float64.  One thread per
// (m, c), c = blockIdx.y; the 2N grid has fewer than 2^31 points (checked at set-up).
__global__ void k_accum_all(const float2* __restrict__ Q, int C, int D, int nb0, int nb1, int nb2, int64_t Nb,
                            double* __restrict__ R) {
    const unsigned m = blockIdx.x * blockDim.x + threadIdx.x;
    if ((int64_t)m >= Nb) return;
    const int c = blockIdx.y;
    const unsigned mneg = neg_index(m, D, (unsigned)nb0, (unsigned)nb1, (unsigned)nb2);
    if (!KP_INB(14, mneg, Nb)) return;
    ff32 acc = {0.f, 0.f};
    for (int d = 0; d < c; ++d)
        acc = ff_add(acc, ff_abs2(Q[(size_t)(d * C - d * (d - 1) / 2 + c - d) * Nb + mneg]));
    const size_t p0 = (size_t)(c * C - c * (c - 1) / 2);
    for (int d = c; d < C; ++d) acc = ff_add(acc, ff_abs2(Q[(p0 + d - c) * Nb + m]));
    R[(size_t)c * Nb + m] = ff_to_double(acc);
}

// r_c = R_c / Nb for the coils c0 .. c0 + nc - 1 (grid c - c0 of out).
__global__ void k_R_to_c(const double* __restrict__ R, int64_t Nb, int nc, double inv_nb, float2* __restrict__ out) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m < Nb * nc) out[m] = make_float2((float)(R[m] * inv_nb), 0.f);
}

// v[j] = r[(j - n) mod 2n] * h[j] on the centred 2N image (lag k_d = j_d - n_d).
// (blockIdx.y selects the coil of a batch: r and v advance by Nb per coil)
__global__ void k_rh(const float2* __restrict__ r, const float2* __restrict__ h, int D, int nb0, int nb1, int nb2,
                     int64_t Nb, float2* __restrict__ v) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Nb) return;
    r += (size_t)blockIdx.y * Nb;
    v += (size_t)blockIdx.y * Nb;
    const int nb[3] = {nb0, nb1, nb2};
    unsigned rr = (unsigned)j, ri = 0, stride = 1;     // the 2N grid has fewer than 2^31 points
    for (int d = D - 1; d >= 0; --d) {
        const unsigned jd = rr % (unsigned)nb[d];
        rr /= (unsigned)nb[d];
        const int k = (int)jd - nb[d] / 2;
        const unsigned idx = (unsigned)(k < 0 ? k + nb[d] : k);
        ri += idx * stride;
        stride *= (unsigned)nb[d];
    }
    if (KP_INB(14, ri, Nb)) v[j] = cmul(r[ri], h[j]);
}

template <typename MT>
__global__ void k_coil_norm2(const MT* __restrict__ maps, int64_t N, int C, double* __restrict__ out) {
    __shared__ double ws[32];
    const int c = blockIdx.y;
    double s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        float2 v = ldc<MT>(maps, (size_t)c * N + i);
        s += (double)v.x * v.x + (double)v.y * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = s;
    __syncthreads();
    if (w == 0) {
        s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) atomicAdd(&out[c], s);
    }
}

__global__ void k_set_norm(double* out, int C, double v) {
    int c = threadIdx.x;
    if (c < C) out[c] = v;
}

// Final step of the fast route: for each sorted sample s of the 2N plan, the denominator
// den = (2^D N)^{-1/2} Re sum_taps phi(t - k) Vhat[k mod g] (type-2 interpolation of the 2N
// plan's forward grid spectrum Vhat = FFT(pad(v_c / Phi))), the taps' products and their sum
// taken in float64, and p[c][perm[s]] = ||s_c||^2 / (2^D den) for the coils c_first ..
// c_first + c_count - 1.  A denominator that is not positive (interpolation error) gives p = 0
// and is counted in *bad.
template <int D>
__global__ void k_den_p(const float2* __restrict__ Vhat, const int* __restrict__ k0t, const float* __restrict__ wt,
                        const int* __restrict__ perm, Geom g2, const double* __restrict__ norm, int cnorm,
                        int c_first, int c_count, float* __restrict__ p, int* __restrict__ bad) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g2.M) return;
    int off[D][KW];                 // the 2N plan's grid has fewer than 2^31 points
    float w[D][KW];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        int stride = 1;
        for (int e = d + 1; e < D; ++e) stride *= g2.g[e];
        const int k0 = k0t[(int64_t)d * g2.M + s];
#pragma unroll
        for (int j = 0; j < KW; ++j) {
            int ix = k0 + j;
            if (ix >= g2.g[d]) ix -= g2.g[d];
            off[d][j] = ix * stride;
            w[d][j] = wt[(int64_t)(d * KW + j) * g2.M + s];
        }
    }
    // sum over the taps of w_a w_b (w_e) Re(Vhat) in float-float: the products of two float32
    // weights are exact, each further product and every addition keeps about 48 bits
    ff32 acc = {0.f, 0.f};
#pragma unroll
    for (int a = 0; a < KW; ++a)
#pragma unroll
        for (int b = 0; b < KW; ++b) {
            const ff32 wab = ff_two_prod(w[0][a], w[1 % D][b]);
            if (D == 2) {
                const int ix = off[0][a] + off[1 % D][b];
                acc = ff_add(acc, ff_mul(wab, KP_INB(15, ix, g2.G) ? Vhat[ix].x : 0.f));
            } else {
#pragma unroll
                for (int e = 0; e < KW; ++e) {
                    const int ix = off[0][a] + off[1 % D][b] + off[D - 1][e];
                    acc = ff_add(acc, ff_mul(ff_mul(wab, w[D - 1][e]), KP_INB(15, ix, g2.G) ? Vhat[ix].x : 0.f));
                }
            }
        }
    const double dv = ff_to_double(acc) * (double)(1 << D) / sqrt((double)g2.N);
    const int64_t i = perm[s];
    if (!KP_INB(15, i, g2.M)) return;
    float val;
    if (dv > 0 && isfinite(dv)) {
        val = (float)(norm[cnorm] / dv);
    } else {
        val = 0.f;
        atomicAdd(bad, 1);
    }
    for (int c = c_first; c < c_first + c_count; ++c) p[(size_t)c * g2.M + i] = val;
}

// ---------------------------------------------------------------- App. B circulant preconditioner
// P = argmin over circulant P of ||A^H A - P||_F^2, P[m, n] = c[(m - n) mod N] (per axis):
//   c[k] = 1/N sum over s in {0, 1}^D of r[k - s N] h[k - s N],  k_d in [0, N_d),
//   r[d] = N^{-1/2} sum_c sum_{m - n = d} s_c^*[m] s_c[n]   (conjugate of IFFT(sum_c |FFT(s_c)|^2) on the 2N grid),
//   h    = the point-spread function of Sec. 5.1 (type-1 NUFFT of ones at 2 f_j on the 2N image).
// The 1/N is the average over the N entries of a circulant diagonal (the printed closed form
// omits it; a uniform scale).  The eigenvalues of P are the DFT of c.

// v[b][m] = s_{c0 + b}[j] with pixel j placed at the origin corner of the 2N grid (lags do not
// depend on the placement), 0 elsewhere.
template <typename MT>
__global__ void k_pad_maps(const MT* __restrict__ maps, int c0, int nc, Geom geo, int D, int nb0, int nb1, int nb2,
                           int64_t Nb, float2* __restrict__ v) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Nb) return;
    const int nb[3] = {nb0, nb1, nb2};
    int64_t r = m, j = 0;
    bool inside = true;
    int ii[MAXD];
    for (int d = D - 1; d >= 0; --d) { ii[d] = (int)(r % nb[d]); r /= nb[d]; }
    for (int d = 0; d < D; ++d) {
        if (ii[d] >= geo.n[d]) inside = false;
        j = j * geo.n[d] + (inside ? ii[d] : 0);
    }
    for (int b = 0; b < nc; ++b)
        v[(size_t)b * Nb + m] = inside ? ldc<MT>(maps, (size_t)(c0 + b) * geo.N + j) : make_float2(0.f, 0.f);
}

// R[m] += sum_b |V_b[m]|^2 (float64)
__global__ void k_accum_abs2(const float2* __restrict__ V, int nc, int64_t Nb, double* __restrict__ R) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Nb) return;
    double acc = R[m];
    for (int b = 0; b < nc; ++b) {
        const float2 a = V[(size_t)b * Nb + m];
        acc = fma((double)a.x, (double)a.x, acc);
        acc = fma((double)a.y, (double)a.y, acc);
    }
    R[m] = acc;
}

// c[k] = scale sum over s in {0,1}^D of conj(rho[(k - s N) mod 2N]) h[k - s N + N]; rho the
// normalised inverse FFT of R (uncentred 2N grid), h centred on the 2N image.
__global__ void k_circ_fold(const float2* __restrict__ rho, const float2* __restrict__ h, Geom geo, int D,
                            int nb0, int nb1, int nb2, float scale, float2* __restrict__ c) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= geo.N) return;
    const int nb[3] = {nb0, nb1, nb2};
    int kk[MAXD];
    int64_t r = k;
    for (int d = D - 1; d >= 0; --d) { kk[d] = (int)(r % geo.n[d]); r /= geo.n[d]; }
    double ax = 0, ay = 0;
    for (int s = 0; s < (1 << D); ++s) {
        int64_t ri = 0, hi = 0;
        for (int d = 0; d < D; ++d) {
            const int lag = kk[d] - (((s >> d) & 1) ? geo.n[d] : 0);     // in [-N_d, N_d)
            ri = ri * nb[d] + (lag < 0 ? lag + nb[d] : lag);
            hi = hi * nb[d] + (lag + geo.n[d]);
        }
        const float2 a = rho[ri], b = h[hi];
        // conj(a) * b
        ax += (double)a.x * b.x + (double)a.y * b.y;
        ay += (double)a.x * b.y - (double)a.y * b.x;
    }
    c[k] = make_float2((float)(ax * scale), (float)(ay * scale));
}

__global__ void k_real_part(const float2* __restrict__ in, int64_t n, float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i].x;
}

kp_status ensure_fft_img(kp_plan p) {
    if (p->fft_img_ok) return KP_OK;
    const Geom& g = p->geo;
    int dims[3] = {g.n[0], g.n[1], g.n[2]};
    KP_TRY_CUFFT(cufftPlanMany(&p->fft_img, g.D, dims, nullptr, 1, (int)g.N, nullptr, 1, (int)g.N, CUFFT_C2C, 1));
    p->fft_img_ok = true;
    return KP_OK;
}

}  // namespace kp

using namespace kp;

kp_status kp::circulant_enqueue(kp_plan plan, cudaStream_t st) {
    if (!plan->traj_set || !plan->maps_set) { set_error("trajectory and maps must be set"); return KP_EINVAL; }
    if (plan->unit_maps) { set_error("not available on an internal plan"); return KP_EINVAL; }
    KP_TRY(pre_create(plan, st));
    KP_TRY(ensure_fft_img(plan));
    PrePlan* q = plan->pre;
    kp_plan nu = plan->pre_nufft;
    const Geom& g = plan->geo;
    if (!plan->d_circ) KP_TRY_CUDA(cudaMalloc(&plan->d_circ, g.N * sizeof(float2)));
    if (!plan->d_circ_eig) KP_TRY_CUDA(cudaMalloc(&plan->d_circ_eig, g.N * sizeof(float)));
    if (q->traj_version != plan->traj_version) {
        KP_TRY(set_trajectory_internal(nu, plan->d_f, 2.0f, st));
        q->traj_version = plan->traj_version;
    }
    KP_TRY_CUFFT(cufftSetStream(q->fft_one, st));
    KP_TRY_CUFFT(cufftSetStream(q->fft_coils, st));
    KP_TRY_CUFFT(cufftSetStream(plan->fft_img, st));
    // R = sum_c |FFT(pad(s_c))|^2 on the 2N grid, batch by batch of coils
    KP_TRY_CUDA(cudaMemsetAsync(q->d_R, 0, (size_t)q->Nb * sizeof(double), st));
    for (int c0 = 0; c0 < g.C; c0 += q->Cb) {
        const int nc = g.C - c0 < q->Cb ? g.C - c0 : q->Cb;
        switch (plan->maps_t) {
            case KP_C64: k_pad_maps<float2><<<nblk(q->Nb, 256), 256, 0, st>>>((const float2*)plan->d_maps, c0, nc, g, g.D, q->nb[0], q->nb[1], q->nb[2], q->Nb, q->d_v); break;
            case KP_C32_BF16: k_pad_maps<__nv_bfloat162><<<nblk(q->Nb, 256), 256, 0, st>>>((const __nv_bfloat162*)plan->d_maps, c0, nc, g, g.D, q->nb[0], q->nb[1], q->nb[2], q->Nb, q->d_v); break;
            default: k_pad_maps<__half2><<<nblk(q->Nb, 256), 256, 0, st>>>((const __half2*)plan->d_maps, c0, nc, g, g.D, q->nb[0], q->nb[1], q->nb[2], q->Nb, q->d_v); break;
        }
        KP_LAUNCH_CHECK();
        if (nc == q->Cb) KP_TRY_CUFFT(cufftExecC2C(q->fft_coils, (cufftComplex*)q->d_v, (cufftComplex*)q->d_v, CUFFT_FORWARD));
        else for (int b = 0; b < nc; ++b)
            KP_TRY_CUFFT(cufftExecC2C(q->fft_one, (cufftComplex*)(q->d_v + (size_t)b * q->Nb), (cufftComplex*)(q->d_v + (size_t)b * q->Nb), CUFFT_FORWARD));
        k_accum_abs2<<<nblk(q->Nb, 256), 256, 0, st>>>(q->d_v, nc, q->Nb, q->d_R);
        KP_LAUNCH_CHECK();
        plan->launches += 2;
    }
    // rho = IFFT(R) / Nb
    k_R_to_c<<<nblk(q->Nb, 256), 256, 0, st>>>(q->d_R, q->Nb, 1, 1.0 / (double)q->Nb, q->d_r);
    KP_LAUNCH_CHECK();
    KP_TRY_CUFFT(cufftExecC2C(q->fft_one, (cufftComplex*)q->d_r, (cufftComplex*)q->d_r, CUFFT_INVERSE));
    // h on the 2N image: the 2N plan's adjoint carries (2^D N)^{-1/2}, h carries N^{-1/2}
    KP_TRY(fill_image(nu->d_kt, nu->geo.M, make_float2(1.f, 0.f), st));
    KP_TRY(adjoint_to_grid(nu, nu->d_kt, KP_C64, nullptr, st));
    KP_TRY(grid_to_image(nu, q->d_h, st));
    // c[k] = 1/N sum r h, r = conj(rho) / sqrt(N), h = 2^{D/2} x (the 2N adjoint of ones)
    const double scale = std::pow(2.0, 0.5 * g.D) / ((double)g.N * std::sqrt((double)g.N));
    k_circ_fold<<<nblk(g.N, 256), 256, 0, st>>>(q->d_r, q->d_h, g, g.D, q->nb[0], q->nb[1], q->nb[2], (float)scale, plan->d_circ);
    KP_LAUNCH_CHECK();
    // eigenvalues: the N-point DFT of c (real for the Hermitian P)
    KP_TRY_CUFFT(cufftExecC2C(plan->fft_img, (cufftComplex*)plan->d_circ, (cufftComplex*)q->d_v, CUFFT_FORWARD));
    k_real_part<<<nblk(g.N, 256), 256, 0, st>>>(q->d_v, g.N, plan->d_circ_eig);
    KP_LAUNCH_CHECK();
    plan->launches += 4;
    plan->circ_ok = true;
    plan->circ_version = plan->traj_version;
    return KP_OK;
}

// Enqueues the whole construction on st without waiting; the number of non-positive
// denominators (entries set to 0) is left in d_flag[7].
kp_status kp::make_preconditioner_enqueue(kp_plan plan, int multichannel, float* p_dev, cudaStream_t st) {
    KP_PHASE("preconditioner");
    if (!plan || !p_dev) { set_error("null argument"); return KP_EINVAL; }
    if (!plan->traj_set || (multichannel && !plan->maps_set)) { set_error("trajectory (and maps) must be set"); return KP_EINVAL; }
    if (plan->unit_maps) { set_error("not available on an internal plan"); return KP_EINVAL; }
    KP_TRY(pre_create(plan, st));
    PrePlan* q = plan->pre;
    kp_plan nu = plan->pre_nufft;
    const Geom& g = plan->geo;
    const bool mc = multichannel != 0;
    const int C = mc ? g.C : 1;
    if (q->traj_version != plan->traj_version) {
        KP_TRY(set_trajectory_internal(nu, plan->d_f, 2.0f, st));
        q->traj_version = plan->traj_version;
    }
    // ||s_c||^2
    if (mc) {
        KP_TRY_CUDA(cudaMemsetAsync(q->d_norm, 0, C * sizeof(double), st));
        dim3 grid(64, C);
        switch (plan->maps_t) {
            case KP_C64: k_coil_norm2<float2><<<grid, 256, 0, st>>>((const float2*)plan->d_maps, g.N, C, q->d_norm); break;
            case KP_C32_BF16: k_coil_norm2<__nv_bfloat162><<<grid, 256, 0, st>>>((const __nv_bfloat162*)plan->d_maps, g.N, C, q->d_norm); break;
            default: k_coil_norm2<__half2><<<grid, 256, 0, st>>>((const __half2*)plan->d_maps, g.N, C, q->d_norm); break;
        }
    } else {
        k_set_norm<<<1, 32, 0, st>>>(q->d_norm, 1, (double)g.N);
    }
    KP_LAUNCH_CHECK();
    plan->launches += 1;
    // R_c = sum_d |FFT(q_cd)|^2
    KP_TRY_CUFFT(cufftSetStream(q->fft_pairs, st));
    KP_TRY_CUFFT(cufftSetStream(q->fft_one, st));
    KP_TRY_CUFFT(cufftSetStream(q->fft_coils, st));
    const int npairs = mc ? q->npairs : 1;
    const bool all_at_once = mc && npairs == q->B && npairs > 1;
    if (!all_at_once) KP_TRY_CUDA(cudaMemsetAsync(q->d_R, 0, (size_t)C * q->Nb * sizeof(double), st));
    for (int p0 = 0; p0 < npairs; p0 += q->B) {
        const int nv = npairs - p0 < q->B ? npairs - p0 : q->B;
        const int nwrite = nv == 1 ? 1 : q->B;      // a lone pair goes through the batch-1 plan
        switch (mc ? plan->maps_t : KP_C64) {
            case KP_C64:
                k_make_q<float2><<<nblk(q->Nb, 256), 256, 0, st>>>(mc ? (const float2*)plan->d_maps : nullptr, q->d_pairs, p0, nv, g,
                                                                   g.D, q->nb[0], q->nb[1], q->nb[2], q->Nb, nwrite, q->d_q);
                break;
            case KP_C32_BF16:
                k_make_q<__nv_bfloat162><<<nblk(q->Nb, 256), 256, 0, st>>>((const __nv_bfloat162*)plan->d_maps, q->d_pairs, p0, nv, g,
                                                                           g.D, q->nb[0], q->nb[1], q->nb[2], q->Nb, nwrite, q->d_q);
                break;
            default:
                k_make_q<__half2><<<nblk(q->Nb, 256), 256, 0, st>>>((const __half2*)plan->d_maps, q->d_pairs, p0, nv, g,
                                                                    g.D, q->nb[0], q->nb[1], q->nb[2], q->Nb, nwrite, q->d_q);
                break;
        }
        KP_LAUNCH_CHECK();
        if (q->f3) {
            // the products are zero outside the image band of the 2N grid (k_make_q's placement)
            KP_TRY(fft3_forward_geo(q->f3, pre_geo(q, g, nwrite, false), q->d_q, q->d_q, plan->launches, st));
        } else {
            KP_TRY_CUFFT(cufftExecC2C(nwrite == 1 ? q->fft_one : q->fft_pairs, (cufftComplex*)q->d_q, (cufftComplex*)q->d_q,
                                      CUFFT_FORWARD));
        }
        if (all_at_once)
            k_accum_all<<<dim3(nblk(q->Nb, 256), C), 256, 0, st>>>(q->d_q, C, g.D, q->nb[0], q->nb[1], q->nb[2], q->Nb,
                                                                   q->d_R);
        else
            k_accum_R<<<nblk(q->Nb, 256), 256, 0, st>>>(q->d_q, q->d_pairs, p0, nv, g.D, q->nb[0], q->nb[1], q->nb[2],
                                                        q->Nb, q->d_R, !mc);
        KP_LAUNCH_CHECK();
        plan->launches += 2;
    }
    // h = adjoint NUFFT of ones on the 2N image
    KP_TRY(fill_image(nu->d_kt, nu->geo.M, make_float2(1.f, 0.f), st));
    plan->launches += 1;
    KP_TRY(adjoint_to_grid(nu, nu->d_kt, KP_C64, nullptr, st));
    KP_TRY(grid_to_image(nu, q->d_h, st));
    KP_TRY_CUDA(cudaMemsetAsync(plan->d_flag + 7, 0, sizeof(int), st));
    // per batch of Cb coils: r_c = IFFT(R_c) / Nb, v_c = r_c * h; then per coil the forward
    // NUFFT of v_c and p_c
    for (int c0 = 0; c0 < C; c0 += q->Cb) {
        const int nc = C - c0 < q->Cb ? C - c0 : q->Cb;
        k_R_to_c<<<nblk(q->Nb * nc, 256), 256, 0, st>>>(q->d_R + (size_t)c0 * q->Nb, q->Nb, nc, 1.0 / (double)q->Nb, q->d_r);
        KP_LAUNCH_CHECK();
        if (q->f3) KP_TRY(fft3_inverse_geo(q->f3, pre_geo(q, g, nc, true), q->d_r, plan->launches, st));   // every lag
        else KP_TRY_CUFFT(cufftExecC2C(nc == 1 ? q->fft_one : q->fft_coils, (cufftComplex*)q->d_r, (cufftComplex*)q->d_r,
                                       CUFFT_INVERSE));
        k_rh<<<dim3(nblk(q->Nb, 256), nc), 256, 0, st>>>(q->d_r, q->d_h, g.D, q->nb[0], q->nb[1], q->nb[2], q->Nb, q->d_v);
        KP_LAUNCH_CHECK();
        plan->launches += 2;
        for (int c = c0; c < c0 + nc; ++c) {
            KP_TRY(forward_grid_only(nu, q->d_v + (size_t)(c - c0) * q->Nb, st));
            if (g.D == 2)
                k_den_p<2><<<nblk(g.M, 256), 256, 0, st>>>(nu->d_gridF, nu->d_k0, nu->d_wt, nu->d_perm, nu->geo, q->d_norm,
                                                           c, mc ? c : 0, mc ? 1 : g.C, p_dev, plan->d_flag + 7);
            else
                k_den_p<3><<<nblk(g.M, 256), 256, 0, st>>>(nu->d_gridF, nu->d_k0, nu->d_wt, nu->d_perm, nu->geo, q->d_norm,
                                                           c, mc ? c : 0, mc ? 1 : g.C, p_dev, plan->d_flag + 7);
            KP_LAUNCH_CHECK();
            plan->launches += 1;
        }
    }
    return KP_OK;
}

extern "C" kp_status kp_make_preconditioner(kp_plan plan, int multichannel, float* p_dev, void* stream) {
    KP_RANGE("kp_make_preconditioner");
    cudaStream_t st = (cudaStream_t)stream;
    KP_TRY(kp::make_preconditioner_enqueue(plan, multichannel, p_dev, st));
    int bad = 0;
    KP_TRY_CUDA(cudaMemcpyAsync(&bad, plan->d_flag + 7, sizeof(int), cudaMemcpyDeviceToHost, st));
    KP_TRY_CUDA(cudaStreamSynchronize(st));
    if (bad) {
        set_error(std::to_string(bad) + " preconditioner denominators were not positive (set to 0)");
        return KP_ENONFINITE;
    }
    return KP_OK;
}
