// Streaming kernels of one relaxation: the free-set scan of eq. active_set
// (Section 5.2) with the fused KKT residual of the stopping rule (Section 8,
// eq. subgradient1), order-preserving compaction of the free pairs, the
// per-pair data of the CD sweep and the sparse sums of the line search
// (Section 6.1.2).  All reductions are deterministic: per-row or per-block
// partials in a fixed order, then one CTA combines them in a fixed order.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "glasso_internal.h"

namespace glx {
namespace {

constexpr int CBLK = 1024;         // candidates per block of the candidate scan
constexpr int RED_T = 256;

__device__ __forceinline__ double sgnd(double x) { return (double)((x > 0.0) - (x < 0.0)); }
__device__ __forceinline__ double soft(double x, double t) {
    double ax = fabs(x) - t;
    return ax > 0.0 ? copysign(ax, x) : 0.0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exclusive block scan of one value per thread (blockDim.x <= 1024).
__device__ long long block_exclusive_scan(long long v, long long *total) {
    __shared__ long long wsum[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        long long s = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) wsum[lane] = s;  // inclusive prefix of warp sums
    }
    __syncthreads();
    long long before = (wid > 0 ? wsum[wid - 1] : 0) + x - v;
    if (total) *total = wsum[((blockDim.x + 31) >> 5) - 1];
    __syncthreads();
    return before;
}

// ---------------------------------------------------------------- full scan
// Three passes over the upper triangle (j >= i) for the free set of
// eq. active_set:
//  1. k_scan_tiles: 64 x 64 tiles, one CTA per tile (tile (b, c), c >= b,
//     band-major).  Each warp takes 8 rows of its tile, a lane two adjacent
//     columns; S, W and A are read with 16-byte loads when n is even and the
//     matrices 16-byte aligned (every row then starts on a 16-byte boundary),
//     every load of a 4-row batch issued
//     before any is used.  The free test runs on FP32 images of S and W built
//     from the high words of the doubles by integer operations (20 mantissa
//     bits); only an entry whose |G_ij| lies within the images' error band of
//     lambda takes the exact FP64 test, so the FP64 pipe (slow on this GPU)
//     stays idle on almost every entry.  A_ij != 0 is read from the bits.
//     Writes the bit masks of free entries per row and 32-column word and the
//     per-row free counts (integer atomics, so the order does not matter).
//  2. k_scan_offsets: one CTA, exclusive scan of the row counts.
//  3. k_scan_emit: one warp per row, 32 mask words at a time (integer work
//     only): writes the free pairs in row-major order.
//  4. k_scan_sums: over the compacted pairs, every lane busy: |S - W| on
//     them and the sums -- the KKT residual of eq. subgradient1 with its max,
//     tr(SA), ||A||_1, nnz(A) (off-diagonal pairs count twice by symmetry).
//     In mode 0 every entry with a nonzero term (A_ij != 0 or |G_ij| >
//     lambda) is a free pair, so these sums are exact; mode 1 (the initial
//     set {|S_ij| > lambda} u supp(A)) gives exact tr(SA), ||A||_1 and nnz
//     only.  Per-CTA partials; the last CTA reduces them in CTA order
//     (deterministic).  The FP64 pipe runs at 1/64 of the FP32 rate on this
//     GPU and costs a warp's issue whatever its active lanes, hence the
//     separate dense pass.
constexpr int ST = 64;                  // tile edge (columns and rows)
constexpr int ST_WARPS = 8;             // warps per tile CTA
constexpr int ST_ROWS = ST / ST_WARPS;  // rows per warp, in batches of ST_BATCH
constexpr int ST_BATCH = 4;
constexpr int EMIT_WARPS = 8;

// FP32 image of x from its high word: sign, rebased exponent, the top 20
// mantissa bits (truncated: relative error below 2^-20).  |x| < 2^-126 maps
// to a signed zero (absolute error below 2^-126), |x| >= 2^128 to infinity.
__device__ __forceinline__ float hi_image(double x) {
    const int hi = __double2hiint(x);
    const int e = ((hi >> 20) & 0x7ff) - 896;
    const unsigned sgn = (unsigned)hi & 0x80000000u;
    const unsigned bits = sgn | ((unsigned)e << 23) | (((unsigned)hi & 0xfffffu) << 3);
    return __uint_as_float(e <= 0 ? sgn : (e >= 255 ? (sgn | 0x7f800000u) : bits));
}

// Bit k of x (k < 16) to bit 2k.
__device__ __forceinline__ unsigned spread16(unsigned x) {
    x &= 0xffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

// Is (s, w, a) free?  |g - g~| <= 2^-20 (|s| + |w|) + 2^-125 + 2^-23 |g~| for
// the images' difference g~ (truncation of both images, one FP32 rounding);
// the band below takes each term twice.  lam_lo <= lambda <= lam_hi are FP32.
__device__ __forceinline__ bool entry_free(double s, double w, double a, double lam, float lam_lo,
                                           float lam_hi, int mode) {
    const bool nz = (((unsigned)__double2hiint(a) & 0x7fffffffu) | (unsigned)__double2loint(a)) != 0u;
    if (nz) return true;
    const float sf = hi_image(s);
    const float x = mode == 0 ? fabsf(sf - hi_image(w)) : fabsf(sf);
    const float band = mode == 0 ? 0x1p-19f * (fabsf(sf) + fabsf(hi_image(w))) + 0x1p-22f * x + 0x1p-100f
                                 : 0x1p-19f * x + 0x1p-100f;
    if (x - band > lam_hi) return true;   // certainly above lambda (NaN: false)
    if (x + band < lam_lo) return false;  // certainly at most lambda
    return mode == 0 ? fabs(s - w) > lam : fabs(s) > lam;  // the border: exact FP64 test
}

template <bool VEC>
__global__ void __launch_bounds__(32 * ST_WARPS) k_scan_tiles(
    const double *__restrict__ S, const double *__restrict__ W, const double *__restrict__ A,
    int64_t n, double lam, float lam_lo, float lam_hi, int mode, uint32_t *__restrict__ mask,
    unsigned long long *__restrict__ rowcnt) {
    const int64_t nb = (n + ST - 1) / ST, nw = (n + 31) / 32;
    // tile t -> (band b, column tile c >= b); band b holds nb - b tiles and
    // starts at t0(b) = b nb - b (b - 1) / 2
    const int64_t t = blockIdx.x;
    const float q = (float)(2 * nb + 1);
    int64_t b = (int64_t)((q - sqrtf(fmaxf(q * q - 8.f * (float)t, 0.f))) * 0.5f);
    b = lmax(0, lmin(b, nb - 1));
    while (b > 0 && b * nb - b * (b - 1) / 2 > t) --b;
    while (b + 1 < nb && (b + 1) * nb - (b + 1) * b / 2 <= t) ++b;
    const int64_t c = b + (t - (b * nb - b * (b - 1) / 2));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t j0 = c * ST + 2 * lane;
#pragma unroll
    for (int bt = 0; bt < ST_ROWS; bt += ST_BATCH) {
        double sv[ST_BATCH][2], wv[ST_BATCH][2], av[ST_BATCH][2];
#pragma unroll
        for (int r = 0; r < ST_BATCH; ++r) {
            const int64_t i = b * ST + warp * ST_ROWS + bt + r;
            const int64_t off = i * n + j0;
            sv[r][0] = sv[r][1] = wv[r][0] = wv[r][1] = av[r][0] = av[r][1] = 0.0;
            if (i < n && j0 + 1 >= i && j0 < n) {
                if (VEC) {  // n even: j0 + 1 < n as well
                    const double2 s2 = __ldg(reinterpret_cast<const double2 *>(S + off));
                    const double2 w2 = __ldg(reinterpret_cast<const double2 *>(W + off));
                    const double2 a2 = __ldg(reinterpret_cast<const double2 *>(A + off));
                    sv[r][0] = s2.x; sv[r][1] = s2.y;
                    wv[r][0] = w2.x; wv[r][1] = w2.y;
                    av[r][0] = a2.x; av[r][1] = a2.y;
                } else {
                    sv[r][0] = __ldg(S + off); wv[r][0] = __ldg(W + off); av[r][0] = __ldg(A + off);
                    if (j0 + 1 < n) {
                        sv[r][1] = __ldg(S + off + 1); wv[r][1] = __ldg(W + off + 1);
                        av[r][1] = __ldg(A + off + 1);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < ST_BATCH; ++r) {
            const int64_t i = b * ST + warp * ST_ROWS + bt + r;
            if (i >= n) break;  // warp-uniform
            bool f[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int64_t j = j0 + e;
                f[e] = j >= i && j < n && entry_free(sv[r][e], wv[r][e], av[r][e], lam, lam_lo, lam_hi, mode);
            }
            const unsigned m0 = __ballot_sync(0xffffffffu, f[0]);
            const unsigned m1 = __ballot_sync(0xffffffffu, f[1]);
            const unsigned w0 = spread16(m0) | (spread16(m1) << 1);
            const unsigned w1 = spread16(m0 >> 16) | (spread16(m1 >> 16) << 1);
            const int64_t wd = c * 2;
            if (lane == 0) {
                mask[i * nw + wd] = w0;
                if (wd + 1 < nw) mask[i * nw + wd + 1] = w1;
                const unsigned cnt = __popc(w0) + __popc(w1);
                if (cnt) atomicAdd(rowcnt + i, (unsigned long long)cnt);
            }
        }
    }
}

// One CTA: exclusive scan of the row counts in place (total at rowcnt[n]
// and in sc->count).
__global__ void __launch_bounds__(1024) k_scan_offsets(unsigned long long *__restrict__ rowcnt,
                                                       int64_t n, DevScalars *sc) {
    const int t = threadIdx.x;
    const int64_t per = (n + 1023) / 1024;
    const int64_t a = t * per, b = lmin(a + per, n);
    long long local = 0;
    for (int64_t i = a; i < b; ++i) local += (long long)rowcnt[i];
    long long total;
    long long off = block_exclusive_scan(local, &total);
    for (int64_t i = a; i < b; ++i) {
        const long long c = (long long)rowcnt[i];
        rowcnt[i] = (unsigned long long)off;
        off += c;
    }
    if (t == 0) {
        rowcnt[n] = (unsigned long long)total;
        sc->count = total;
    }
}

// Free pairs of each row at the row's offset, row-major.  A warp per row (rows
// strided over the grid's warps); lane l holds mask word w0 + l of the chunk.
__global__ void __launch_bounds__(32 * EMIT_WARPS) k_scan_emit(int64_t n, const uint32_t *__restrict__ mask,
                                                              const unsigned long long *__restrict__ rowoff,
                                                              int32_t *__restrict__ oi,
                                                              int32_t *__restrict__ oj) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (n + 31) / 32;
    const int64_t tw = (int64_t)gridDim.x * EMIT_WARPS;
    for (int64_t i = (int64_t)blockIdx.x * EMIT_WARPS + (threadIdx.x >> 5); i < n; i += tw) {
        long long off = (long long)rowoff[i];
        for (int64_t wb = i / 32; wb < nw; wb += 32) {
            const int64_t w = wb + lane;
            uint32_t m = w < nw ? mask[i * nw + w] : 0u;
            const int cnt = __popc(m);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            long long pos = off + incl - cnt;
            while (m) {
                const int bit = __ffs(m) - 1;
                m &= m - 1u;
                oi[pos] = (int32_t)i;
                oj[pos] = (int32_t)(w * 32 + bit);
                ++pos;
            }
            off += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

constexpr int SUM_T = 128;

// |S - W| on the free pairs and the sums over them (see above); the pair
// count comes from k_scan_offsets.  part: 5 doubles per CTA.
__global__ void __launch_bounds__(SUM_T) k_scan_sums(const double *__restrict__ S, const double *__restrict__ W,
                                                     const double *__restrict__ A, int64_t n, double lam,
                                                     const int32_t *__restrict__ oi,
                                                     const int32_t *__restrict__ oj,
                                                     double *__restrict__ oabsg, double *__restrict__ part,
                                                     DevScalars *sc) {
    __shared__ double red[5][SUM_T];
    __shared__ bool last_s;
    const long long np = sc->count;
    double kkt = 0.0, kmax = 0.0, tr = 0.0, l1 = 0.0, nnz = 0.0;
    for (long long p = (long long)blockIdx.x * SUM_T + threadIdx.x; p < np; p += (long long)gridDim.x * SUM_T) {
        const int64_t i = oi[p], j = oj[p];
        const double s = S[i * n + j], w = W[i * n + j], a = A[i * n + j];
        const double g = s - w, ag = fabs(g);
        if (oabsg) oabsg[p] = ag;
        const bool nz = a != 0.0;
        if (nz || ag > lam) {
            const double wt = (j == i) ? 1.0 : 2.0;
            const double r = nz ? fabs(g + lam * sgnd(a)) : ag - lam;
            kkt += wt * r;
            kmax = fmax(kmax, r);
            if (nz) {
                tr += wt * s * a;
                l1 += wt * fabs(a);
                nnz += wt;
            }
        }
    }
    red[0][threadIdx.x] = kkt;
    red[1][threadIdx.x] = kmax;
    red[2][threadIdx.x] = tr;
    red[3][threadIdx.x] = l1;
    red[4][threadIdx.x] = nnz;
    __syncthreads();
    for (int h = SUM_T / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            red[0][threadIdx.x] += red[0][threadIdx.x + h];
            red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + h]);
            red[2][threadIdx.x] += red[2][threadIdx.x + h];
            red[3][threadIdx.x] += red[3][threadIdx.x + h];
            red[4][threadIdx.x] += red[4][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) part[blockIdx.x * 5 + k] = red[k][0];
        __threadfence();
        last_s = atomicAdd(&sc->scan_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last_s) return;
    // the last CTA: fixed-order reduction of the CTA partials (L2 loads)
    kkt = kmax = tr = l1 = nnz = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += SUM_T) {
        kkt += __ldcg(part + 5 * b);
        kmax = fmax(kmax, __ldcg(part + 5 * b + 1));
        tr += __ldcg(part + 5 * b + 2);
        l1 += __ldcg(part + 5 * b + 3);
        nnz += __ldcg(part + 5 * b + 4);
    }
    red[0][threadIdx.x] = kkt;
    red[1][threadIdx.x] = kmax;
    red[2][threadIdx.x] = tr;
    red[3][threadIdx.x] = l1;
    red[4][threadIdx.x] = nnz;
    __syncthreads();
    for (int h = SUM_T / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            red[0][threadIdx.x] += red[0][threadIdx.x + h];
            red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + h]);
            red[2][threadIdx.x] += red[2][threadIdx.x + h];
            red[3][threadIdx.x] += red[3][threadIdx.x + h];
            red[4][threadIdx.x] += red[4][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sc->kkt_sum = red[0][0];
        sc->kkt_max = red[1][0];
        sc->trSA = red[2][0];
        sc->l1 = red[3][0];
        sc->nnz = (long long)red[4][0];
        sc->scan_done = 0u;  // ready for the next launch
    }
}

// ---------------------------------------------------------------- candidates
__global__ void k_cand_flags(const double *__restrict__ S, const double *__restrict__ W,
                             const double *__restrict__ A, int64_t n, double lam,
                             const int32_t *__restrict__ ci, const int32_t *__restrict__ cj,
                             const uint8_t *__restrict__ tag, int level, int64_t ncand,
                             uint8_t *__restrict__ flags, long long *__restrict__ blkcnt) {
    __shared__ long long wc[32];
    const int64_t base = (int64_t)blockIdx.x * CBLK;
    long long c = 0;
    for (int r = threadIdx.x; r < CBLK; r += blockDim.x) {
        const int64_t p = base + r;
        uint8_t f = 0;
        if (p < ncand && (tag == nullptr || tag[p] >= level)) {
            const int64_t i = ci[p], j = cj[p];
            const double g = S[i * n + j] - W[i * n + j];
            f = (A[i * n + j] != 0.0) || (fabs(g) > lam);
        }
        if (p < ncand) flags[p] = f;
        c += f;
    }
    c = warp_sum_ll(c);
    if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wc[w];
        blkcnt[blockIdx.x] = s;
    }
}

// Exclusive scan of nb block counts in one CTA; total to sc->count.
__global__ void __launch_bounds__(1024) k_blk_scan(long long *__restrict__ blkcnt, int64_t nb,
                                                   DevScalars *sc) {
    const int t = threadIdx.x;
    const int64_t per = (nb + 1023) / 1024;
    const int64_t a = t * per, b = lmin(a + per, nb);
    long long local = 0;
    for (int64_t k = a; k < b; ++k) local += blkcnt[k];
    long long total;
    long long off = block_exclusive_scan(local, &total);
    for (int64_t k = a; k < b; ++k) {
        long long c = blkcnt[k];
        blkcnt[k] = off;
        off += c;
    }
    if (t == 0) sc->count = total;
}

__global__ void __launch_bounds__(CBLK) k_cand_write(const double *__restrict__ S,
                                                     const double *__restrict__ W, int64_t n,
                                                     const int32_t *__restrict__ ci,
                                                     const int32_t *__restrict__ cj,
                                                     int64_t ncand, const uint8_t *__restrict__ flags,
                                                     const long long *__restrict__ blkoff,
                                                     int32_t *__restrict__ oi, int32_t *__restrict__ oj,
                                                     double *__restrict__ oabsg) {
    const int64_t p = (int64_t)blockIdx.x * CBLK + threadIdx.x;
    const long long f = (p < ncand) ? flags[p] : 0;
    long long off = block_exclusive_scan(f, nullptr);
    if (f) {
        const long long pos = blkoff[blockIdx.x] + off;
        const int64_t i = ci[p], j = cj[p];
        oi[pos] = (int32_t)i;
        oj[pos] = (int32_t)j;
        if (oabsg) oabsg[pos] = fabs(S[i * n + j] - W[i * n + j]);
    }
}

// ---------------------------------------------------------------- misc
__global__ void k_support(const double *__restrict__ A, int64_t n, const int32_t *__restrict__ fi,
                          const int32_t *__restrict__ fj, int64_t nf, uint8_t *__restrict__ flag) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nf;
         p += (int64_t)gridDim.x * blockDim.x)
        flag[p] = A[(int64_t)fi[p] * n + fj[p]] != 0.0;
}

__global__ void k_init_diag(const double *__restrict__ S, int64_t n, double lam,
                            double *__restrict__ A, DevScalars *sc) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double d = S[i * n + i] + lam;
        if (!(d > 0.0)) atomicExch(&sc->err, 1);
        A[i * n + i] = 1.0 / d;
    }
}

// max_{i < j} |S_ij| (the smallest lambda whose minimiser is diagonal), for
// the continuation schedule.  One row per block step, coalesced along the
// row; block maximum by warp shuffles; one atomicMax per block on the bits of
// the (non-negative) double, whose unsigned order is the numeric order.
// sc->smax_bits must be zero on entry.
__global__ void k_offdiag_absmax(const double *__restrict__ S, int64_t n, DevScalars *sc) {
    __shared__ double red[8];
    double m = 0.0;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const double *row = S + i * n;
        for (int64_t j = i + 1 + threadIdx.x; j < n; j += blockDim.x) m = fmax(m, fabs(row[j]));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m = fmax(m, red[k]);
        atomicMax(&sc->smax_bits, (unsigned long long)__double_as_longlong(m));
    }
}

__global__ void k_pair_prep(const double *__restrict__ S, const double *__restrict__ W,
                            const double *__restrict__ A, int64_t n, const int32_t *__restrict__ pi,
                            const int32_t *__restrict__ pj, int64_t np, double *__restrict__ inva,
                            double *__restrict__ g, double *__restrict__ aval,
                            double *__restrict__ sval) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = pi[p], j = pj[p];
        const double wij = W[i * n + j];
        const double a = (i == j) ? wij * wij : wij * wij + W[i * n + i] * W[j * n + j];
        inva[p] = 1.0 / a;
        g[p] = S[i * n + j] - wij;
        aval[p] = A[i * n + j];
        sval[p] = S[i * n + j];
    }
}

// Per-block partial sums over pairs: what = 0: delta, trSD, moved;
// what = 1: dl1 at alpha.
__global__ void k_pair_sums(const double *__restrict__ g, const double *__restrict__ aval,
                            const double *__restrict__ sval, const double *__restrict__ D,
                            const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                            int64_t np, double lam, double alpha, int what,
                            double *__restrict__ part) {
    __shared__ double red[3][RED_T];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)RED_T + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * RED_T) {
        const double mult = (pi[p] == pj[p]) ? 1.0 : 2.0;
        const double d = D[p], a = aval[p];
        if (what == 0) {
            s0 += mult * (g[p] * d + lam * (fabs(a + d) - fabs(a)));
            s1 += mult * sval[p] * d;
            s2 += (d != 0.0) ? 1.0 : 0.0;
        } else {
            s0 += mult * (fabs(a + alpha * d) - fabs(a));
        }
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    red[2][threadIdx.x] = s2;
    __syncthreads();
    for (int w = RED_T / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
            red[2][threadIdx.x] += red[2][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x * 3 + 0] = red[0][0];
        part[blockIdx.x * 3 + 1] = red[1][0];
        part[blockIdx.x * 3 + 2] = red[2][0];
    }
}

__global__ void k_pair_sums_final(const double *__restrict__ part, int nblk, int what,
                                  DevScalars *sc) {
    if (threadIdx.x != 0) return;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int b = 0; b < nblk; ++b) {
        s0 += part[b * 3 + 0];
        s1 += part[b * 3 + 1];
        s2 += part[b * 3 + 2];
    }
    if (what == 0) {
        sc->delta = s0;
        sc->trSD = s1;
        sc->moved = s2 > 0.0;
    } else {
        sc->dl1 = s0;
    }
}

__global__ void k_scatter_pairs(double *__restrict__ T, int64_t n, const int32_t *__restrict__ pi,
                                const int32_t *__restrict__ pj, const double *__restrict__ aval,
                                const double *__restrict__ D, int64_t np, double alpha) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = pi[p], j = pj[p];
        const double v = aval[p] + alpha * D[p];
        T[i * n + j] = v;
        T[j * n + i] = v;
    }
}

inline unsigned grid_for(int64_t work, int per = 256) {
    int64_t g = (work + per - 1) / per;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (unsigned)g;
}

}  // namespace

// FP32 bounds lam_lo <= lam <= lam_hi.
static void lam_bounds(double lam, float &lo, float &hi) {
    lo = hi = (float)lam;
    if ((double)lo > lam) lo = nextafterf(lo, -INFINITY);
    if ((double)hi < lam) hi = nextafterf(hi, INFINITY);
}

static unsigned sums_grid(int64_t n) { return (unsigned)lmax(8, lmin(152, n / 32)); }

// The four passes of the full scan (see above) on scratch mask (n x ceil(n/32)
// words), rowcnt (n + 1) and part (5 x sums_grid(n) doubles).
static cudaError_t scan_full_on(const double *S, const double *W, const double *A, int64_t n, double lam,
                                int mode, uint32_t *mask, unsigned long long *rowcnt, double *part,
                                int32_t *oi, int32_t *oj, double *oabsg, DevScalars *sc, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(rowcnt, 0, (size_t)(n + 1) * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    float lo, hi;
    lam_bounds(lam, lo, hi);
    const int64_t nb = (n + ST - 1) / ST;
    const unsigned tiles = (unsigned)(nb * (nb + 1) / 2);
    // 16-byte loads need every row start on a 16-byte boundary
    const bool vec = n % 2 == 0 && (((uintptr_t)S | (uintptr_t)W | (uintptr_t)A) & 15u) == 0;
    if (vec)
        k_scan_tiles<true><<<tiles, 32 * ST_WARPS, 0, st>>>(S, W, A, n, lam, lo, hi, mode, mask, rowcnt);
    else
        k_scan_tiles<false><<<tiles, 32 * ST_WARPS, 0, st>>>(S, W, A, n, lam, lo, hi, mode, mask, rowcnt);
    k_scan_offsets<<<1, 1024, 0, st>>>(rowcnt, n, sc);
    const unsigned ge = (unsigned)lmin((n + EMIT_WARPS - 1) / EMIT_WARPS, 152 * 4);
    k_scan_emit<<<ge, 32 * EMIT_WARPS, 0, st>>>(n, mask, rowcnt, oi, oj);
    k_scan_sums<<<sums_grid(n), SUM_T, 0, st>>>(S, W, A, n, lam, oi, oj, oabsg, part, sc);
    counted(4);
    return cudaGetLastError();
}

cudaError_t scan_full(const double *S, const double *W, const double *A, int64_t n, double lam,
                      int mode, Work &w, int32_t *oi, int32_t *oj, double *oabsg, DevScalars *sc,
                      cudaStream_t st) {
    static_assert(sizeof(long long) == sizeof(unsigned long long), "row counts");
    return scan_full_on(S, W, A, n, lam, mode, w.mask, reinterpret_cast<unsigned long long *>(w.rowcnt),
                        w.rowred, oi, oj, oabsg, sc, st);
}

cudaError_t scan_cand(const double *S, const double *W, const double *A, int64_t n, double lam,
                      const int32_t *ci, const int32_t *cj, const uint8_t *tag, int level,
                      int64_t ncand, Work &w, int32_t *oi, int32_t *oj, double *oabsg,
                      DevScalars *sc, cudaStream_t st) {
    if (ncand <= 0) return cudaMemsetAsync(&sc->count, 0, sizeof(long long), st);
    const int64_t nb = (ncand + CBLK - 1) / CBLK;
    if (nb > w.cap_blk) return cudaErrorInvalidValue;
    k_cand_flags<<<(unsigned)nb, 256, 0, st>>>(S, W, A, n, lam, ci, cj, tag, level, ncand,
                                               w.flags, w.blkcnt);
    counted(1);
    k_blk_scan<<<1, 1024, 0, st>>>(w.blkcnt, nb, sc);
    counted(1);
    k_cand_write<<<(unsigned)nb, CBLK, 0, st>>>(S, W, n, ci, cj, ncand, w.flags, w.blkcnt, oi,
                                                oj, oabsg);
    counted(1);
    return cudaGetLastError();
}

cudaError_t support_flags(const double *A, int64_t n, const int32_t *fi, const int32_t *fj,
                          int64_t nf, uint8_t *flag, cudaStream_t st) {
    k_support<<<grid_for(nf), 256, 0, st>>>(A, n, fi, fj, nf, flag);
    counted(1);
    return cudaGetLastError();
}

cudaError_t offdiag_absmax(const double *S, int64_t n, DevScalars *sc, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(&sc->smax_bits, 0, sizeof(sc->smax_bits), st);
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)std::min<int64_t>(std::max<int64_t>(n, 1), 152 * 8);
    k_offdiag_absmax<<<g, 256, 0, st>>>(S, n, sc);
    counted(1);
    return cudaGetLastError();
}

cudaError_t init_diag(const double *S, int64_t n, double lam, double *A, DevScalars *sc,
                      cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(A, 0, (size_t)(n * n) * sizeof(double), st);
    if (e != cudaSuccess) return e;
    k_init_diag<<<grid_for(n), 256, 0, st>>>(S, n, lam, A, sc);
    counted(1);
    return cudaGetLastError();
}

cudaError_t pair_prep(const double *S, const double *W, const double *A, int64_t n, double lam,
                      const int32_t *pi, const int32_t *pj, int64_t np, double *inva, double *g,
                      double *aval, double *sval, cudaStream_t st) {
    (void)lam;
    if (np <= 0) return cudaSuccess;
    k_pair_prep<<<grid_for(np), 256, 0, st>>>(S, W, A, n, pi, pj, np, inva, g, aval, sval);
    counted(1);
    return cudaGetLastError();
}

static cudaError_t pair_sums(const double *g, const double *aval, const double *sval,
                             const double *D, const int32_t *pi, const int32_t *pj, int64_t np,
                             double lam, double alpha, int what, Work &w, DevScalars *sc,
                             cudaStream_t st) {
    int nblk = (int)lmin((np + RED_T - 1) / RED_T, 1024);
    if (nblk < 1) nblk = 1;
    if (3 * nblk > w.cap_red) return cudaErrorInvalidValue;
    k_pair_sums<<<nblk, RED_T, 0, st>>>(g, aval, sval, D, pi, pj, np, lam, alpha, what, w.redbuf);
    counted(1);
    k_pair_sums_final<<<1, 32, 0, st>>>(w.redbuf, nblk, what, sc);
    counted(1);
    return cudaGetLastError();
}

cudaError_t ls_delta(const double *g, const double *aval, const double *sval, const double *D,
                     const int32_t *pi, const int32_t *pj, int64_t np, double lam, Work &w,
                     DevScalars *sc, cudaStream_t st) {
    return pair_sums(g, aval, sval, D, pi, pj, np, lam, 0.0, 0, w, sc, st);
}

cudaError_t ls_dl1(const double *aval, const double *D, const int32_t *pi, const int32_t *pj,
                   int64_t np, double alpha, Work &w, DevScalars *sc, cudaStream_t st) {
    return pair_sums(aval, aval, aval, D, pi, pj, np, 0.0, alpha, 1, w, sc, st);
}

cudaError_t ls_build_trial(const double *A, double *T, int64_t n, const int32_t *pi,
                           const int32_t *pj, const double *aval, const double *D, int64_t np,
                           double alpha, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(T, A, (size_t)(n * n) * sizeof(double),
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    if (np > 0) {
        k_scatter_pairs<<<grid_for(np), 256, 0, st>>>(T, n, pi, pj, aval, D, np, alpha);
        counted(1);
    }
    return cudaGetLastError();
}

cudaError_t ls_apply(double *A, int64_t n, const int32_t *pi, const int32_t *pj,
                     const double *aval, const double *D, int64_t np, double alpha,
                     cudaStream_t st) {
    if (np > 0) {
        k_scatter_pairs<<<grid_for(np), 256, 0, st>>>(A, n, pi, pj, aval, D, np, alpha);
        counted(1);
    }
    return cudaGetLastError();
}

}  // namespace glx

// ============================================================================
// Allocation-free variant of the full free-set scan (glasso_free_set_noalloc).
//
// Some callers cannot allocate device memory: code that runs under another
// framework's memory manager (which owns the whole device heap), or a
// latency-critical loop that cannot take cudaMalloc's implicit device-wide
// synchronisation.  This entry point gives them the level-0 free-set scan
// with its scratch (row bit masks, row counts and partial sums, result
// scalars) in one file-scope device array of fixed size, so it needs no
// context and allocates nothing.  Every GPU that loads the library holds the
// array until the process exits.
namespace glx {
namespace {

constexpr int64_t NA_N = GLASSO_NOALLOC_MAX_N;
constexpr size_t na_round(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t NA_MASK_OFF = 0;
constexpr size_t NA_MASK_BYTES = na_round(sizeof(uint32_t) * NA_N * ((NA_N + 31) / 32));
constexpr size_t NA_CNT_OFF = NA_MASK_OFF + NA_MASK_BYTES;
constexpr size_t NA_CNT_BYTES = na_round(sizeof(long long) * (NA_N + 1));
constexpr size_t NA_RED_OFF = NA_CNT_OFF + NA_CNT_BYTES;
constexpr size_t NA_RED_BYTES = na_round(sizeof(double) * 6 * NA_N);
constexpr size_t NA_SC_OFF = NA_RED_OFF + NA_RED_BYTES;
constexpr size_t NA_TOTAL = NA_SC_OFF + na_round(sizeof(DevScalars));

// The scratch itself.  In host code this name is only a host-side stand-in;
// the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_na_scratch[NA_TOTAL];

constexpr int NA_MAX_DEV = 64;
std::mutex g_na_mu;
unsigned char *g_na_ptr[NA_MAX_DEV] = {nullptr};

// Set-up, once per device, with that device current: look up the device
// address of the scratch array.
cudaError_t na_scratch(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEV) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = (unsigned char *)p;
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace glx

extern "C" glasso_status glasso_free_set_noalloc(const double *S, const double *W,
                                                 const double *A, int64_t n, double lambda,
                                                 int32_t *out_i, int32_t *out_j, double *absg,
                                                 int64_t *count, double *rel_kkt,
                                                 double *max_kkt, void *stream) {
    using namespace glx;
    if (!S || !W || !A || !out_i || !out_j || !count || n < 1 || !(lambda > 0.0) ||
        !isfinite(lambda))
        return GLASSO_EINVAL;
    if (n > GLASSO_NOALLOC_MAX_N) return GLASSO_EINVAL;  // beyond the fixed scratch
    unsigned char *base = nullptr;
    if (na_scratch(&base) != cudaSuccess) return GLASSO_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *mask = (uint32_t *)(base + NA_MASK_OFF);
    long long *rowcnt = (long long *)(base + NA_CNT_OFF);
    double *rowred = (double *)(base + NA_RED_OFF);
    DevScalars *sc = (DevScalars *)(base + NA_SC_OFF);
    // Every mask word and partial sum the scan reads is written by it first,
    // and the row counts are cleared by the scan itself; the result scalars
    // (and the sums pass's completion counter) are cleared here, so that no
    // value of the previous call can leak into this one.
    if (cudaMemsetAsync(sc, 0, sizeof(DevScalars), st) != cudaSuccess) return GLASSO_ECUDA;
    static_assert(5 * 152 * sizeof(double) <= NA_RED_BYTES, "partials of the sums pass");
    if (scan_full_on(S, W, A, n, lambda, 0, mask, reinterpret_cast<unsigned long long *>(rowcnt), rowred,
                     out_i, out_j, absg, sc, st) != cudaSuccess)
        return GLASSO_ECUDA;
    if (cudaGetLastError() != cudaSuccess) return GLASSO_ECUDA;
    DevScalars h;
    if (cudaMemcpyAsync(&h, sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return GLASSO_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GLASSO_ECUDA;
    *count = h.count;
    if (rel_kkt) *rel_kkt = h.kkt_sum / h.l1;
    if (max_kkt) *max_kkt = h.kkt_max;
    return GLASSO_OK;
}
