// Streaming kernels of one relaxation: the free-set scan of eq. active_set
// (Section 5.2) with the fused KKT residual of the stopping rule (Section 8,
// eq. subgradient1), order-preserving compaction of the free pairs, the
// per-pair data of the CD sweep and the sparse sums of the line search
// (Section 6.1.2).  All reductions are deterministic: per-row or per-block
// partials in a fixed order, then one CTA combines them in a fixed order.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "glasso_internal.h"

namespace glx {
namespace {

constexpr int SCAN_WARPS = 8;      // rows per CTA of the full scan
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
// One warp per row i covers the upper part j >= i.  Writes the ballot masks
// of free entries, the per-row free count, and per-row partial sums of the
// KKT residual, tr(SA), ||A||_1 and nnz(A) over the full matrix (off-diagonal
// entries count twice by symmetry).
__global__ void k_scan_rows(const double *__restrict__ S, const double *__restrict__ W,
                            const double *__restrict__ A, int64_t n, double lam, int mode,
                            uint32_t *__restrict__ mask, long long *__restrict__ rowcnt,
                            double *__restrict__ rowred) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * SCAN_WARPS + (threadIdx.x >> 5);
    if (i >= n) return;
    const int64_t nw = (n + 31) / 32;
    long long cnt = 0;
    double kkt = 0.0, kmax = 0.0, tr = 0.0, l1 = 0.0, nnz = 0.0;
    const double *Si = S + i * n, *Wi = W + i * n, *Ai = A + i * n;
    for (int64_t jb = i & ~(int64_t)31; jb < n; jb += 32) {
        const int64_t j = jb + lane;
        const bool valid = j >= i && j < n;
        bool fr = false;
        if (valid) {
            const double s = Si[j], w = Wi[j], a = Ai[j];
            const double g = s - w, ag = fabs(g);
            const bool nz = a != 0.0;
            fr = nz || (mode == 0 ? ag > lam : fabs(s) > lam);
            // most entries have A_ij = 0 and |G_ij| <= lambda and add nothing:
            // keep the FP64 work (slow on this GPU) to the rest
            if (nz || ag > lam) {
                const double wt = (j == i) ? 1.0 : 2.0;
                const double r = nz ? g + lam * sgnd(a) : soft(g, lam);
                kkt += wt * fabs(r);
                kmax = fmax(kmax, fabs(r));
                if (nz) {
                    tr += wt * s * a;
                    l1 += wt * fabs(a);
                    nnz += wt;
                }
            }
        }
        const uint32_t m = __ballot_sync(0xffffffffu, fr);
        if (lane == 0) mask[i * nw + jb / 32] = m;
        cnt += __popc(m);
    }
    kkt = warp_sum(kkt);
    kmax = warp_max(kmax);
    tr = warp_sum(tr);
    l1 = warp_sum(l1);
    nnz = warp_sum(nnz);
    if (lane == 0) {
        rowcnt[i] = cnt;
        double *r = rowred + i * 6;
        r[0] = kkt;
        r[1] = kmax;
        r[2] = tr;
        r[3] = l1;
        r[4] = nnz;
    }
}

// One CTA: exclusive scan of the row counts (in place; total at rowcnt[n]) and
// the fixed-order reduction of the row partial sums into the scalars.
__global__ void __launch_bounds__(1024) k_scan_finish(long long *__restrict__ rowcnt,
                                                      const double *__restrict__ rowred,
                                                      int64_t n, DevScalars *sc, int sums) {
    __shared__ double red[5][1024];
    const int t = threadIdx.x;
    const int64_t per = (n + 1023) / 1024;
    const int64_t a = t * per, b = lmin(a + per, n);
    long long local = 0;
    double kkt = 0.0, kmax = 0.0, tr = 0.0, l1 = 0.0, nnz = 0.0;
    for (int64_t i = a; i < b; ++i) {
        local += rowcnt[i];
        if (sums) {
            const double *r = rowred + i * 6;
            kkt += r[0];
            kmax = fmax(kmax, r[1]);
            tr += r[2];
            l1 += r[3];
            nnz += r[4];
        }
    }
    long long total;
    long long off = block_exclusive_scan(local, &total);
    for (int64_t i = a; i < b; ++i) {
        long long c = rowcnt[i];
        rowcnt[i] = off;
        off += c;
    }
    if (t == 0) {
        rowcnt[n] = total;
        sc->count = total;
    }
    if (!sums) return;
    red[0][t] = kkt;
    red[1][t] = kmax;
    red[2][t] = tr;
    red[3][t] = l1;
    red[4][t] = nnz;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (t < w) {
            red[0][t] += red[0][t + w];
            red[1][t] = fmax(red[1][t], red[1][t + w]);
            red[2][t] += red[2][t + w];
            red[3][t] += red[3][t + w];
            red[4][t] += red[4][t + w];
        }
        __syncthreads();
    }
    if (t == 0) {
        sc->kkt_sum = red[0][0];
        sc->kkt_max = red[1][0];
        sc->trSA = red[2][0];
        sc->l1 = red[3][0];
        sc->nnz = (long long)red[4][0];
    }
}

// Writes the free pairs of each row at the row's offset, in row-major order.
__global__ void k_scan_write(const double *__restrict__ S, const double *__restrict__ W, int64_t n,
                             const uint32_t *__restrict__ mask, const long long *__restrict__ rowoff,
                             int32_t *__restrict__ oi, int32_t *__restrict__ oj,
                             double *__restrict__ oabsg) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * SCAN_WARPS + (threadIdx.x >> 5);
    if (i >= n) return;
    const int64_t nw = (n + 31) / 32;
    long long off = rowoff[i];
    for (int64_t w = i / 32; w < nw; ++w) {
        const uint32_t m = mask[i * nw + w];
        if (m & (1u << lane)) {
            const long long pos = off + __popc(m & ((1u << lane) - 1u));
            const int64_t j = w * 32 + lane;
            oi[pos] = (int32_t)i;
            oj[pos] = (int32_t)j;
            if (oabsg) oabsg[pos] = fabs(S[i * n + j] - W[i * n + j]);
        }
        off += __popc(m);
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

cudaError_t scan_full(const double *S, const double *W, const double *A, int64_t n, double lam,
                      int mode, Work &w, int32_t *oi, int32_t *oj, double *oabsg, DevScalars *sc,
                      cudaStream_t st) {
    const unsigned g = (unsigned)((n + SCAN_WARPS - 1) / SCAN_WARPS);
    k_scan_rows<<<g, 32 * SCAN_WARPS, 0, st>>>(S, W, A, n, lam, mode, w.mask, w.rowcnt, w.rowred);
    counted(1);
    k_scan_finish<<<1, 1024, 0, st>>>(w.rowcnt, w.rowred, n, sc, 1);
    counted(1);
    k_scan_write<<<g, 32 * SCAN_WARPS, 0, st>>>(S, W, n, w.mask, w.rowcnt, oi, oj, oabsg);
    counted(1);
    return cudaGetLastError();
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
    // Every mask word, row count and partial sum the scan reads is written by
    // it first; only the result scalars are cleared, so that no value of the
    // previous call can leak into this one.
    if (cudaMemsetAsync(sc, 0, sizeof(DevScalars), st) != cudaSuccess) return GLASSO_ECUDA;
    const unsigned g = (unsigned)((n + SCAN_WARPS - 1) / SCAN_WARPS);
    k_scan_rows<<<g, 32 * SCAN_WARPS, 0, st>>>(S, W, A, n, lambda, 0, mask, rowcnt, rowred);
    k_scan_finish<<<1, 1024, 0, st>>>(rowcnt, rowred, n, sc, 1);
    k_scan_write<<<g, 32 * SCAN_WARPS, 0, st>>>(S, W, n, mask, rowcnt, out_i, out_j, absg);
    counted(3);
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
