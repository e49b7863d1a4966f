// PCD-CG: the Jacobi-parallel Newton-direction solver (Section 2, eq.
// IST_direction with D = the diagonal of the Hessian, accelerated by
// non-linear conjugate gradients as in Section 6.3) for the restricted Newton
// LASSO of eq. Quad_MLE_l1_prior, the alternative to the sequential CD sweep.
//
// One iteration on the free pairs p = (i, j), i <= j (w_p = 2 off the
// diagonal, 1 on it; a_p = W_ij^2 + W_ii W_jj, or W_ii^2 on the diagonal):
//   b_p = G_p + (W Delta W)_p,   c_p = A_p + Delta_p,
//   d_p = S_{lambda/a_p}(c_p - b_p/a_p) - c_p            (every coordinate's own 1-D minimiser)
//   beta = max(0, <d, d - d_prev>_w / <d_prev, d_prev>_w) (Polak-Ribiere-plus; 0 at the start)
//   P = d + beta P_prev, or d when that is not a descent direction
//   t = argmin_{t >= 0} t g1 + t^2 g2 / 2 + lambda sum_p w_p (|c_p + t P_p| - |c_p|),
//       g1 = <b, P>_w,  g2 = <P, W P W>_w                 (exact, piecewise quadratic)
//   Delta += t P, with exact zeros where the minimiser is a kink of the
//   coordinate and where a coordinate whose own minimiser is zero can no
//   longer be moved (the zero snap).
// Stops when d = 0, after `iters` iterations, once max|d| <= rtol max|d| of
// the first iteration (Section 8 runs the inner solver to relative precision
// 1e-4), or when the step is 0.
//
// GPU form.  The only O(n) per pair work is (W P W) on the pairs: an SpMM
// V = P W over the symmetric CSR pattern of the pairs, written transposed
// (Vt = V^T, rows contiguous), then one dot per pair of row i of W with row j
// of Vt (an SDDMM).  b is carried from iteration to iteration: b += t (W P W)
// plus, for the few coordinates set to an exact zero, the same two passes on
// their corrections, so (W Delta W) is never recomputed from U = Delta W;
// U is formed once at the end (SpMM of the final Delta).  All iterations run
// in one cooperative launch (k_pcd_persist): every CTA owns a fixed slice of
// the pairs, the phases are separated by grid barriers, and each CTA reduces
// the per-CTA partials itself in CTA order, so every CTA takes the same
// scalar decision (stop, CG coefficient, descent, the step) without another
// barrier.  The kink walk runs in CTA 0.  At the precision stop the
// coordinates whose own minimiser is zero take their exact zero (the final
// shrinkage).
//
// Exact step: phi'(t) = g1 + g2 t + h(t), h(t+) = lambda sum_p w_p P_p
// sign(c_p + t P_p) (sign(P_p) at a kink), is nondecreasing, so the minimiser
// lies in [0, t0], t0 = -(g1 + h(0+)) / g2.  The kinks t_p = -c_p / P_p in
// (L, R] = (0, t0] are counted; while they exceed what one CTA sorts in
// shared memory the interval is halved by the sign of phi'(mid+); then they
// are sorted and walked in increasing order from h(L+).
#include <math.h>

#include <algorithm>

#include "glasso_internal.h"

namespace glx {
namespace {

constexpr int PT = 512;           // threads of a CTA of the persistent kernel
constexpr int PW = PT / 32;       // its warps
constexpr int KCAP = 4096;        // kinks sorted in shared memory
constexpr int SP_ROWS = 32;       // rows of V per SpMM CTA
constexpr int SP_COLS = 128;      // columns of V per SpMM CTA
constexpr int PCD_MAX_G = 160;    // CTAs of the persistent kernel, at most (one per SM)
// warp groups of the persistent SpMM: as many tiles in flight as fit the shared memory
template <typename T>
constexpr int SPLIT_NH = sizeof(T) == 4 ? 4 : 2;

struct PcdState {
    int done;        // the stopping rule fired
    int it;          // iterations completed
    int nk;          // kinks gathered in (0, R]
    unsigned tctr[2];  // SpMM tiles handed out (alternating between SpMM phases)
    int err;         // a bounded grid-barrier wait expired
    unsigned bar;    // grid barrier arrivals
    int pad;
    double d0max;    // max |d| of the first iteration
    double t, kinkt; // the step (from CTA 0's walk)
};

__device__ __forceinline__ double sgnd(double x) { return (double)((x > 0.0) - (x < 0.0)); }
__device__ __forceinline__ double soft(double x, double th) {
    const double ax = fabs(x) - th;
    return ax > 0.0 ? copysign(ax, x) : 0.0;
}

// Block-wide sum over the CTA (every thread gets the result).
__device__ double block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) x += red[w];
        red[32] = x;
    }
    __syncthreads();
    return red[32];
}

// ---------------------------------------------------------------- CSR of the pairs
// Row r lists every pair touching r: (r, j) for pairs (r, j) and (r, i) for
// pairs (i, r), i < r, as (column, pair index); rows are sorted by column so
// the SpMM sums in a fixed order.
__global__ void k_csr_count(const int32_t *__restrict__ pi, const int32_t *__restrict__ pj, int64_t np,
                            int *__restrict__ cnt) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        atomicAdd(cnt + pi[p], 1);
        if (pi[p] != pj[p]) atomicAdd(cnt + pj[p], 1);
    }
}

// One CTA: exclusive scan of cnt (n) into ptr (n + 1); cursor = a copy.
__global__ void __launch_bounds__(1024) k_csr_scan(const int *__restrict__ cnt, int64_t n,
                                                 int *__restrict__ ptr, int *__restrict__ cursor) {
    __shared__ int wsum[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int64_t per = (n + 1023) / 1024, a = t * per, b = lmin(a + per, n);
    int local = 0;
    for (int64_t r = a; r < b; ++r) local += cnt[r];
    int x = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    int off = (wid > 0 ? wsum[wid - 1] : 0) + x - local;
    for (int64_t r = a; r < b; ++r) {
        ptr[r] = off;
        cursor[r] = off;
        off += cnt[r];
    }
    if (t == 1023) ptr[n] = off;
}

__global__ void k_csr_fill(const int32_t *__restrict__ pi, const int32_t *__restrict__ pj, int64_t np,
                           int *__restrict__ cursor, int *__restrict__ col, int *__restrict__ pid) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int i = pi[p], j = pj[p];
        int q = atomicAdd(cursor + i, 1);
        col[q] = j;
        pid[q] = (int)p;
        if (i != j) {
            q = atomicAdd(cursor + j, 1);
            col[q] = i;
            pid[q] = (int)p;
        }
    }
}

// Insertion sort of each row by column (rows are short: the pairs per row).
__global__ void k_csr_sort(const int *__restrict__ ptr, int64_t n, int *__restrict__ col,
                           int *__restrict__ pid) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int a = ptr[r], b = ptr[r + 1];
        for (int q = a + 1; q < b; ++q) {
            const int c = col[q], d = pid[q];
            int k = q - 1;
            while (k >= a && col[k] > c) {
                col[k + 1] = col[k];
                pid[k + 1] = pid[k];
                --k;
            }
            col[k + 1] = c;
            pid[k + 1] = d;
        }
    }
}

// The CSR positions of each pair's entries: qi[p] in row pi[p], qj[p] in row
// pj[p] (the same entry for a diagonal pair).
__global__ void k_csr_pos(const int *__restrict__ ptr, int64_t n, const int *__restrict__ col,
                          const int *__restrict__ pid, const int32_t *__restrict__ pi,
                          const int32_t *__restrict__ pj, int *__restrict__ qi, int *__restrict__ qj) {
    const int64_t nq = ptr[n];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int p = pid[q];
        if (col[q] == pj[p]) {  // the entry in row pi[p]
            qi[p] = (int)q;
            if (pi[p] == pj[p]) qj[p] = (int)q;
        } else {
            qj[p] = (int)q;
        }
    }
}

// ---------------------------------------------------------------- (W X W) on the pairs
// V = X W for the symmetric X given on the pairs (values x, CSR pattern):
// V_r = sum over the row's entries of x W_col.  A tile is a 32 x 128 block of
// V, formed by one CTA (rows over its warps, columns over the lanes, every
// load a coalesced row segment of W) in shared memory and written out either
// transposed (TRANS: out = V^T, 32 consecutive elements per warp store) or as
// is.  Zero values are skipped.  Tiles are taken from `first` in steps of
// `step` (a grid-stride loop).
template <typename T, bool TRANS>
__device__ __noinline__ void spmm_tiles(const T *__restrict__ W, int64_t n, const int *__restrict__ ptr,
                           const int *__restrict__ col, const int *__restrict__ pid,
                           const double *__restrict__ x, const double *__restrict__ vq, T *__restrict__ out,
                           int64_t first, int64_t step, T (*tile)[SP_COLS + 1]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int64_t tr = (n + SP_ROWS - 1) / SP_ROWS, tc = (n + SP_COLS - 1) / SP_COLS;
    for (int64_t tt = first; tt < tr * tc; tt += step) {
        const int64_t r0 = (tt / tc) * SP_ROWS, k0 = (tt % tc) * SP_COLS;
        for (int rl = warp; rl < SP_ROWS; rl += nwarp) {
            const int64_t r = r0 + rl;
            T acc[SP_COLS / 32];
#pragma unroll
            for (int m = 0; m < SP_COLS / 32; ++m) acc[m] = T(0);
            if (r < n) {
                // four entries at a time, all their loads issued before the products
                // (x may come from other CTAs of the launch: read through L2)
                const int qb = ptr[r], qe = ptr[r + 1];
                for (int q0 = qb; q0 < qe; q0 += 4) {
                    T vv[4], wv[4][SP_COLS / 32];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int q = q0 + u;
                        vv[u] = q < qe ? (T)__ldcg(vq ? vq + q : x + pid[q]) : T(0);
                        const T *wr = W + (int64_t)(q < qe ? col[q] : 0) * n + k0 + lane;
#pragma unroll
                        for (int m = 0; m < SP_COLS / 32; ++m)
                            wv[u][m] = (vv[u] != T(0) && k0 + lane + 32 * m < n) ? wr[32 * m] : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int m = 0; m < SP_COLS / 32; ++m) acc[m] = fma(vv[u], wv[u][m], acc[m]);
                }
            }
            if (TRANS) {
#pragma unroll
                for (int m = 0; m < SP_COLS / 32; ++m) tile[rl][lane + 32 * m] = acc[m];
            } else if (r < n) {
#pragma unroll
                for (int m = 0; m < SP_COLS / 32; ++m)
                    if (k0 + lane + 32 * m < n) out[r * n + k0 + lane + 32 * m] = acc[m];
            }
        }
        if (TRANS) {
            __syncthreads();
            for (int c = warp; c < SP_COLS; c += nwarp) {
                const int64_t k = k0 + c;
                if (k >= n) break;
                if (r0 + lane < n) out[k * n + r0 + lane] = tile[lane][c];
            }
            __syncthreads();
        }
    }
}

// The persistent kernel's SpMM: the CTA's warps split into NH groups, each
// forming its own tiles (the CTA's tiles dealt round robin) with its own
// shared-memory tile and named barrier, so NH tiles' load chains overlap.
template <typename T, int NH>
__device__ __noinline__ void spmm_tiles_split(const T *__restrict__ W, int64_t n, const int *__restrict__ ptr,
                                              const int *__restrict__ col, const double *__restrict__ vq,
                                              T *__restrict__ out, unsigned *ctr, unsigned char *smem, int sr) {
    __shared__ unsigned grab[NH];
    const int lane = threadIdx.x & 31, nwh = (blockDim.x >> 5) / NH;  // warps per group
    const int h = (threadIdx.x >> 5) / nwh, warp = (threadIdx.x >> 5) % nwh;
    T(*tile)[SP_COLS + 1] = reinterpret_cast<T(*)[SP_COLS + 1]>(smem) + h * SP_ROWS;
    const unsigned nthr = (unsigned)nwh * 32u;
    const int64_t tr = (n + sr - 1) / sr, tc = (n + SP_COLS - 1) / SP_COLS;
    for (;;) {
        // the next tile, from a counter shared by every group of the grid
        if (warp == 0 && lane == 0) grab[h] = atomicAdd(ctr, 1u);
        asm volatile("bar.sync %0, %1;" ::"r"(1 + h), "r"(nthr) : "memory");
        const int64_t tt = grab[h];
        if (tt >= tr * tc) break;
        const int64_t r0 = (tt / tc) * sr, k0 = (tt % tc) * SP_COLS;
        for (int rl = warp; rl < sr; rl += nwh) {
            const int64_t r = r0 + rl;
            T acc[SP_COLS / 32];
#pragma unroll
            for (int m = 0; m < SP_COLS / 32; ++m) acc[m] = T(0);
            if (r < n) {
                const int qb = ptr[r], qe = ptr[r + 1];
                for (int q0 = qb; q0 < qe; q0 += 4) {
                    T vv[4], wv[4][SP_COLS / 32];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int q = q0 + u;
                        vv[u] = q < qe ? (T)__ldcg(vq + q) : T(0);
                        const T *wr = W + (int64_t)(q < qe ? col[q] : 0) * n + k0 + lane;
#pragma unroll
                        for (int m = 0; m < SP_COLS / 32; ++m)
                            wv[u][m] = (q < qe && k0 + lane + 32 * m < n) ? wr[32 * m] : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int m = 0; m < SP_COLS / 32; ++m) acc[m] = fma(vv[u], wv[u][m], acc[m]);
                }
            }
#pragma unroll
            for (int m = 0; m < SP_COLS / 32; ++m) tile[rl][lane + 32 * m] = acc[m];
        }
        asm volatile("bar.sync %0, %1;" ::"r"(1 + h), "r"(nthr) : "memory");
        for (int c = warp; c < SP_COLS; c += nwh) {
            const int64_t k = k0 + c;
            if (k >= n) break;
            if (lane < sr && r0 + lane < n) out[k * n + r0 + lane] = tile[lane][c];
        }
        asm volatile("bar.sync %0, %1;" ::"r"(1 + h), "r"(nthr) : "memory");
    }
}

// out_p = W_{i,:} . Vt_{j,:} (= (W X W)_ij for Vt = (X W)^T): one warp per pair
// (warps numbered w0, w0 + nw, ...), lanes over the row, sum in T.
template <typename T>
__device__ __noinline__ void sddmm_pairs(const T *__restrict__ W, const T *__restrict__ Vt, int64_t n,
                            const int32_t *__restrict__ pi, const int32_t *__restrict__ pj, int64_t np,
                            double *__restrict__ out, int64_t w0, int64_t nw, const double *__restrict__ P,
                            double *g2) {
    const int lane = threadIdx.x & 31;
    for (int64_t p = w0; p < np; p += nw) {
        const T *a = W + (int64_t)pi[p] * n, *b = Vt + (int64_t)pj[p] * n;
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        int64_t k = lane;
        // four independent sums (Vt may come from other CTAs of the launch: read through L2)
        for (; k + 96 < n; k += 128) {
            const T a0 = a[k], a1 = a[k + 32], a2 = a[k + 64], a3 = a[k + 96];
            const T b0 = __ldcg(b + k), b1 = __ldcg(b + k + 32), b2 = __ldcg(b + k + 64), b3 = __ldcg(b + k + 96);
            s0 = fma(a0, b0, s0);
            s1 = fma(a1, b1, s1);
            s2 = fma(a2, b2, s2);
            s3 = fma(a3, b3, s3);
        }
        for (; k < n; k += 32) s0 = fma(a[k], __ldcg(b + k), s0);
        T s = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            out[p] = (double)s;
            // g2 += w_p P_p (W P W)_p, P from other CTAs of the launch (lane 0 only)
            if (g2) *g2 += (pi[p] == pj[p] ? 1.0 : 2.0) * __ldcg(P + p) * (double)s;
        }
    }
}

// Stand-alone launches (the initial b from a given Delta, the final U).
template <typename T, bool TRANS>
__global__ void __launch_bounds__(256) k_pair_spmm(const T *__restrict__ W, int64_t n,
                                                   const int *__restrict__ ptr, const int *__restrict__ col,
                                                   const int *__restrict__ pid, const double *__restrict__ x,
                                                   T *__restrict__ out) {
    __shared__ T tile[SP_ROWS][SP_COLS + 1];
    spmm_tiles<T, TRANS>(W, n, ptr, col, pid, x, nullptr, out, blockIdx.x, gridDim.x, tile);
}

template <typename T>
__global__ void __launch_bounds__(256) k_pair_sddmm(const T *__restrict__ W, const T *__restrict__ Vt,
                                                    int64_t n, const int32_t *__restrict__ pi,
                                                    const int32_t *__restrict__ pj, int64_t np,
                                                    double *__restrict__ out) {
    sddmm_pairs<T>(W, Vt, n, pi, pj, np, out, (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5),
                   (int64_t)gridDim.x * 8, nullptr, nullptr);
}

__global__ void k_vec_add(double *__restrict__ b, const double *__restrict__ add, int64_t np) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x)
        b[p] += add[p];
}

// ---------------------------------------------------------------- the persistent solver
struct PcdVec {
    const int32_t *pi, *pj;
    const double *inva, *g, *aval;  // 1/a_p, G_p, A_p
    double *D, *b, *c, *d, *dprev, *P, *wpw, *corr, *tmp;
    uint8_t *zt;
    int64_t np;
    double *part;      // 2 x 4 partials per CTA (alternating between reductions)
    double *vq;        // the SpMM's values in CSR entry order (P, or the corrections)
    const int *qi, *qj;  // each pair's two CSR positions
    double *kt, *kj;   // kinks gathered in (0, R]: times and jumps (KCAP)
    int *kp;           //                             pair indices
    int sr;            // rows per SpMM tile (<= SP_ROWS): fewer for a small n, so the grid has tiles to share
};

__device__ __forceinline__ double pair_w(const PcdVec &v, int64_t p) { return v.pi[p] == v.pj[p] ? 1.0 : 2.0; }

__device__ __forceinline__ void red_release(unsigned *p, unsigned x) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(x) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned x;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(x) : "l"(p) : "memory");
    return x;
}

// Grid barrier: a monotonic arrival counter (the k-th barrier completes at
// k G); the wait is bounded (about 2 s of SM cycles) and sets st->err.
__device__ bool pcd_barrier(PcdState *st, unsigned G, unsigned &epoch) {
    __shared__ int ok_s;
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) {
        red_release(&st->bar, 1u);
        const unsigned target = epoch * G;
        int ok = 1;
        const long long t0 = clock64();
        unsigned spins = 0;
        volatile int *verr = &st->err;
        while ((int)(ld_acquire(&st->bar) - target) < 0) {
            if ((++spins & 31u) == 0 && (*verr || clock64() - t0 > 4000000000ll)) {
                ok = 0;
                atomicExch(&st->err, 1);
                break;
            }
        }
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Grid-wide reduction of NV values per thread (slot k a max when bit k of
// maxmask is set, else a sum): CTA partials, a barrier, then every CTA
// combines all partials in CTA order, so all take the same totals.
template <int NV>
__device__ __noinline__ bool grid_reduce(double (&v)[NV], unsigned maxmask, const PcdVec &pv, PcdState *st, unsigned G,
                            unsigned &epoch, unsigned &nred, double *red, double *bc, int nact) {
    // only the first nact warps hold values (the others skip the FP64 shuffles,
    // which cost a warp's issue slots on this GPU whatever the values)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *part = pv.part + (size_t)(nred++ & 1u) * 4 * G;
    if (warp < nact) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const bool mx = (maxmask >> k) & 1u;
            double x = v[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double y = __shfl_xor_sync(0xffffffffu, x, o);
                x = mx ? fmax(x, y) : x + y;
            }
            if (lane == 0) red[k * PW + warp] = x;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const bool mx = (maxmask >> k) & 1u;
            double x = mx ? 0.0 : 0.0;  // every max slot here is of non-negative values
            for (int w = 0; w < nact; ++w) x = mx ? fmax(x, red[k * PW + w]) : x + red[k * PW + w];
            part[blockIdx.x * 4 + k] = x;
        }
    }
    if (!pcd_barrier(st, G, epoch)) return false;
    if (warp == 0) {
        // every partial this lane combines, loaded before any is used (at most
        // PCD_MAX_G / 32 per lane)
        double pv[NV][PCD_MAX_G / 32];
#pragma unroll
        for (int u = 0; u < PCD_MAX_G / 32; ++u) {
            const int b = lane + 32 * u;
#pragma unroll
            for (int k = 0; k < NV; ++k) pv[k][u] = b < (int)G ? __ldcg(part + b * 4 + k) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const bool mx = (maxmask >> k) & 1u;
            double x = mx ? -INFINITY : 0.0;
#pragma unroll
            for (int u = 0; u < PCD_MAX_G / 32; ++u)
                if (lane + 32 * u < (int)G) x = mx ? fmax(x, pv[k][u]) : x + pv[k][u];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double y = __shfl_xor_sync(0xffffffffu, x, o);
                x = mx ? fmax(x, y) : x + y;
            }
            if (lane == 0) bc[k] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = bc[k];
    return true;
}

// lambda sum_p w_p P_p sign(c_p + t P_p) (sign(P_p) where c_p + t P_p = 0) and
// the number of kinks in (L, R], over one thread's share of all pairs (CTA 0's
// fallback for more than KCAP kinks).
__device__ __noinline__ void slope_and_kinks(const PcdVec &v, double lam, double t, double L, double R, double &h,
                                double &cnt) {
    h = 0.0;
    cnt = 0.0;
    for (int64_t p = threadIdx.x; p < v.np; p += blockDim.x) {
        const double P = __ldcg(v.P + p);
        if (P == 0.0) continue;
        const double c = __ldcg(v.c + p), w = pair_w(v, p);
        const double x = c + t * P;
        h += lam * w * P * (x != 0.0 ? sgnd(x) : sgnd(P));
        if (c != 0.0 && sgnd(c) != sgnd(P)) {
            const double tk = -c / P;
            if (tk > L && tk <= R) cnt += 1.0;
        }
    }
}

// The exact step, in CTA 0 (dynamic shared memory: KCAP keys, jumps and pair
// indices): sort the nk kinks of (0, R] gathered by all CTAs and walk them in
// increasing order from h(0+).  When more than KCAP lie in (0, R], the
// interval (L, R] is first halved (bit-pattern bisection on the sign of
// phi'(mid+)) over all pairs until its kinks fit, or until it holds a single
// kink value; they are gathered again and the walk starts from h(L+).
__device__ __noinline__ void pcd_walk(const PcdVec &v, double lam, double g1, double g2, double h0, double R,
                                      int nk, double *key, double *jmp, int *kid, double *red, double &t_out,
                                      double &kink_out) {
    __shared__ int nkink;
    double L = 0.0, HL = h0;
    bool group = false;  // (L, R] holds more than KCAP kinks, all at R
    if (nk <= KCAP) {  // the kinks of (0, R], gathered by all CTAs
        for (int s = threadIdx.x; s < nk; s += blockDim.x) {
            key[s] = __ldcg(v.kt + s);
            jmp[s] = __ldcg(v.kj + s);
            kid[s] = __ldcg(v.kp + s);
        }
        if (threadIdx.x == 0) nkink = nk;
        __syncthreads();
    }
    for (int pass = nk <= KCAP ? 2 : 0; pass < 2; ++pass) {
        if (threadIdx.x == 0) nkink = 0;
        __syncthreads();
        double gjump = 0.0;
        for (int64_t p = threadIdx.x; p < v.np; p += blockDim.x) {
            const double P = __ldcg(v.P + p), c = __ldcg(v.c + p);
            if (P == 0.0 || c == 0.0 || sgnd(c) == sgnd(P)) continue;
            const double tk = -c / P;
            if (!(tk > L && tk <= R)) continue;
            const double j = 2.0 * lam * pair_w(v, p) * fabs(P);
            if (group) {
                gjump += j;
            } else {
                const int s = atomicAdd(&nkink, 1);
                if (s < KCAP) {
                    key[s] = tk;
                    jmp[s] = j;
                    kid[s] = (int)p;
                }
            }
        }
        if (group) {
            gjump = block_sum(gjump, red);
            const double ts = -(g1 + HL) / g2;
            if (ts <= R) {
                t_out = ts;
                kink_out = -1.0;
            } else if (g1 + g2 * R + HL + gjump >= 0.0) {
                t_out = kink_out = R;
            } else {
                t_out = -(g1 + HL + gjump) / g2;
                kink_out = -1.0;
            }
            return;
        }
        __syncthreads();
        if (nkink <= KCAP) break;
        // too many kinks: narrow (L, R], then gather again
        for (int round = 0; round < 70; ++round) {
            const long long lb = __double_as_longlong(L), rb = __double_as_longlong(R);
            const double mid = __longlong_as_double(lb + (rb - lb) / 2);
            if (!(mid > L && mid < R)) {
                group = true;
                break;
            }
            double hm, cm;
            slope_and_kinks(v, lam, mid, mid, mid, hm, cm);
            hm = block_sum(hm, red);
            if (g1 + g2 * mid + hm >= 0.0) {
                R = mid;
            } else {
                L = mid;
                HL = hm;
            }
            double hh, cnt;
            slope_and_kinks(v, lam, L, L, R, hh, cnt);
            cnt = block_sum(cnt, red);
            if (cnt <= (double)KCAP) break;
        }
    }
    const int m = min(nkink, KCAP);
    // bitonic sort of (key, pair index), padded to a power of two
    int m2 = 1;
    while (m2 < m) m2 <<= 1;
    for (int s = m + threadIdx.x; s < m2; s += blockDim.x) {
        key[s] = INFINITY;
        jmp[s] = 0.0;
        kid[s] = 0x7fffffff;
    }
    __syncthreads();
    for (int size = 2; size <= m2; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int s = threadIdx.x; s < m2; s += blockDim.x) {
                const int o = s ^ stride;
                if (o > s) {
                    const bool up = (s & size) == 0;
                    const bool gt = key[s] > key[o] || (key[s] == key[o] && kid[s] > kid[o]);
                    if (gt == up) {
                        const double tk = key[s], tj = jmp[s];
                        const int ti = kid[s];
                        key[s] = key[o]; jmp[s] = jmp[o]; kid[s] = kid[o];
                        key[o] = tk; jmp[o] = tj; kid[o] = ti;
                    }
                }
            }
            __syncthreads();
        }
    // The walk in increasing order from h(L+).  A few kinks (the usual case at
    // n = 2000): every thread takes the same serial steps.  Many (dense free
    // sets): in parallel.  (The serial steps are a dependent FP64 chain: 31 us
    // for 1200 kinks, against 12 us in parallel; below about a hundred kinks
    // the serial walk is the faster.)
    double t = NAN, kinkt = -1.0;
    if (m <= 96) {
        double H = HL;
        int k = 0;
        while (k < m) {
            const double tk = key[k];
            const double ts = -(g1 + H) / g2;
            if (ts <= tk) {
                t = ts;
                break;
            }
            double jump = 0.0;
            int k2 = k;
            while (k2 < m && key[k2] == tk) jump += jmp[k2++];
            if (g1 + g2 * tk + H + jump >= 0.0) {
                t = kinkt = tk;
                break;
            }
            H += jump;
            k = k2;
        }
        if (isnan(t)) t = -(g1 + H) / g2;
    } else {
        // The slope phi'(t) = g1 + g2 t + h(t) rises at each kink group (equal
        // times) by its jumps.  The walk stops
        // at the first group whose slope just right of it is >= 0: inside the
        // smooth piece before it (t = -(g1 + H) / g2, H the jumps before the
        // group) if the slope is already >= 0 just left of it, else on the kink.
        // In parallel: an inclusive scan of the jumps (each thread a contiguous
        // chunk, then the chunks' totals), the first such group by a minimum.
        __shared__ double wsum[PT / 32];
        __shared__ int first;
        const int nt = (int)blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
        const int ch = (m + nt - 1) / nt, c0 = min(m, tid * ch), c1 = min(m, c0 + ch);
        double run = 0.0;
        for (int i = c0; i < c1; ++i) {
            run += jmp[i];
            jmp[i] = run;  // (the chunk's own prefix for now)
        }
        // exclusive prefix of the chunk totals: warp scan, then the warps' totals
        double x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        if (tid == 0) first = 0x7fffffff;
        __syncthreads();
        double woff = 0.0;
        for (int w = 0; w < wid; ++w) woff += wsum[w];
        const double off = woff + (x - run);
        for (int i = c0; i < c1; ++i) jmp[i] += off;  // S_i = jumps up to and including i
        __syncthreads();
        for (int i = c0; i < c1; ++i) {
            if (i + 1 < m && key[i + 1] == key[i]) continue;  // not the group's last kink
            if (g1 + g2 * key[i] + (HL + jmp[i]) >= 0.0) {
                atomicMin(&first, i);
                break;
            }
        }
        __syncthreads();
        if (first == 0x7fffffff) {
            t = -(g1 + (HL + (m > 0 ? jmp[m - 1] : 0.0))) / g2;
        } else {
            int k = first;
            const double tk = key[k];
            while (k > 0 && key[k - 1] == tk) --k;  // the group's first kink
            const double H = HL + (k > 0 ? jmp[k - 1] : 0.0);
            const double ts = -(g1 + H) / g2;
            if (ts <= tk) {
                t = ts;
            } else {
                t = kinkt = tk;
            }
        }
    }
    t_out = t;
    kink_out = kinkt;
}

// All PCD-CG iterations in one cooperative launch (see the top of the file).
// Six grid barriers per iteration: the direction's reduction, the search
// direction's, the SpMM, the SDDMM with g2, the kink gather, and the step
// from CTA 0.  The corrections of an iteration's exact zeros are applied to b
// at the start of the next one (only then are they needed).
template <typename T>
__global__ void __launch_bounds__(PT, 1) k_pcd_persist(const T *__restrict__ W, T *__restrict__ Vt, int64_t n,
                                                        double lam, const int *__restrict__ ptr,
                                                        const int *__restrict__ col, const int *__restrict__ pid,
                                                        PcdVec v, int iters, int cg, double rtol,
                                                        PcdState *st) {
    extern __shared__ __align__(16) unsigned char pcd_smem[];
    __shared__ double red[4 * PW + 8], bc[4];
    const unsigned G = gridDim.x;
    unsigned epoch = 0, nred = 0;
    const int64_t np = v.np;
    const int64_t lo = np * blockIdx.x / G, hi = np * (blockIdx.x + 1) / G;
    const int nact = (int)lmin(PW, (hi - lo + 31) / 32);  // warps holding pairs of this CTA's slice
    const int64_t gw0 = (int64_t)blockIdx.x * PW + (threadIdx.x >> 5), gnw = (int64_t)G * PW;
    // Vt = (X W)^T, X in vq (the tile in the dynamic shared memory, which the walk also uses)
    unsigned nspmm = 0;
    auto spmm = [&]() {
        // tiles handed out by st->tctr[nspmm & 1]; the other counter is cleared
        // by CTA 0 for the next SpMM (which is at least one barrier away)
        unsigned *ctr = &st->tctr[nspmm & 1u];
        spmm_tiles_split<T, SPLIT_NH<T>>(W, n, ptr, col, v.vq, Vt, ctr, pcd_smem, v.sr);
        if (blockIdx.x == 0 && threadIdx.x == 0) st->tctr[(nspmm + 1) & 1u] = 0u;
        ++nspmm;
        __syncthreads();
    };
    int it = 0;
    double d0max = 0.0;
    bool corr_pending = false;  // this thread's pairs got corrections in the last update
    for (;;) {
        if (it >= iters) break;
        // 1. direction, max |d| and the Polak-Ribiere sums (and whether the last
        //    update left corrections of b to apply first)
        double r4[4] = {0.0, 0.0, 0.0, corr_pending ? 1.0 : 0.0};
        auto direction = [&](double (&r)[4]) {
            for (int64_t p = lo + threadIdx.x; p < hi; p += PT) {
                const double c = v.aval[p] + v.D[p];
                const double dp = soft(c - v.b[p] * v.inva[p], lam * v.inva[p]) - c;
                v.c[p] = c;
                v.d[p] = dp;
                r[0] = fmax(r[0], fabs(dp));
                if (cg && it > 0) {
                    const double w = pair_w(v, p), dq = v.dprev[p];
                    r[1] += w * dp * (dp - dq);
                    r[2] += w * dq * dq;
                }
            }
        };
        direction(r4);
        if (!grid_reduce<4>(r4, 9u, v, st, G, epoch, nred, red, bc, nact)) break;
        if (r4[3] != 0.0) {
            // b += (W C W) for the last update's corrections C (in vq), then the
            // direction again
            spmm();
            if (!pcd_barrier(st, G, epoch)) break;
            sddmm_pairs<T>(W, Vt, n, v.pi, v.pj, np, v.tmp, gw0, gnw, nullptr, nullptr);
            if (!pcd_barrier(st, G, epoch)) break;
            for (int64_t p = lo + threadIdx.x; p < hi; p += PT) v.b[p] += __ldcg(v.tmp + p);
            r4[0] = r4[1] = r4[2] = r4[3] = 0.0;
            direction(r4);
            if (!grid_reduce<4>(r4, 9u, v, st, G, epoch, nred, red, bc, nact)) break;
        }
        corr_pending = false;
        const double dmax = r4[0];
        if (dmax == 0.0) break;
        if (it > 0 && rtol > 0.0 && dmax <= rtol * d0max) {
            // the final shrinkage: own minimiser zero -> the exact zero
            for (int64_t p = lo + threadIdx.x; p < hi; p += PT) {
                const double c = v.c[p];
                if (c != 0.0 && c + v.d[p] == 0.0) v.D[p] = -v.aval[p];
            }
            break;
        }
        if (it == 0) d0max = dmax;
        const double beta = (cg && it > 0 && r4[2] > 0.0) ? fmax(0.0, r4[1] / r4[2]) : 0.0;
        // 2. search direction (also into vq for the SpMM), zero flags, g1 and
        //    the l1 slope h(0+)
        double r2[2] = {0.0, 0.0};
        for (int64_t p = lo + threadIdx.x; p < hi; p += PT) {
            const double dp = v.d[p], c = v.c[p];
            const double P = dp + beta * v.P[p];
            v.P[p] = P;
            v.vq[v.qi[p]] = P;
            v.vq[v.qj[p]] = P;
            v.zt[p] = c + dp == 0.0;
            const double w = pair_w(v, p);
            r2[0] += w * v.b[p] * P;
            if (P != 0.0) r2[1] += lam * w * P * (c != 0.0 ? sgnd(c) : sgnd(P));
        }
        if (!grid_reduce<2>(r2, 0u, v, st, G, epoch, nred, red, bc, nact)) break;
        if (beta != 0.0 && r2[0] + r2[1] >= 0.0) {  // not a descent direction: the PCD direction
            r2[0] = r2[1] = 0.0;
            for (int64_t p = lo + threadIdx.x; p < hi; p += PT) {
                const double dp = v.d[p], c = v.c[p], w = pair_w(v, p);
                v.P[p] = dp;
                v.vq[v.qi[p]] = dp;
                v.vq[v.qj[p]] = dp;
                r2[0] += w * v.b[p] * dp;
                if (dp != 0.0) r2[1] += lam * w * dp * (c != 0.0 ? sgnd(c) : sgnd(dp));
            }
            if (!grid_reduce<2>(r2, 0u, v, st, G, epoch, nred, red, bc, nact)) break;
        }
        const double g1 = r2[0], h0 = r2[1];
        // 3. (W P W) on the pairs, and g2 = <P, W P W>_w
        spmm();
        if (!pcd_barrier(st, G, epoch)) break;
        double r1[1] = {0.0};
        sddmm_pairs<T>(W, Vt, n, v.pi, v.pj, np, v.wpw, gw0, gnw, v.P, &r1[0]);
        if (!grid_reduce<1>(r1, 0u, v, st, G, epoch, nred, red, bc, PW)) break;
        const double g2 = r1[0];
        if (!(g2 > 0.0) || g1 + h0 >= 0.0) break;  // a zero step ends the iterations
        const double R = -(g1 + h0) / g2;
        // 4. the kinks t_p = -c_p / P_p in (0, R], gathered by all CTAs (a
        //    division only for the candidates that a product test keeps)
        for (int64_t p = lo + threadIdx.x; p < hi; p += PT) {
            const double P = v.P[p], c = v.c[p];
            if (P == 0.0 || c == 0.0 || sgnd(c) == sgnd(P)) continue;
            if (fabs(c) > R * fabs(P) * (1.0 + 0x1p-40)) continue;
            const double tk = -c / P;
            if (!(tk > 0.0 && tk <= R)) continue;
            const int s = atomicAdd(&st->nk, 1);
            if (s < KCAP) {
                v.kt[s] = tk;
                v.kj[s] = 2.0 * lam * pair_w(v, p) * fabs(P);
                v.kp[s] = (int)p;
            }
        }
        if (!pcd_barrier(st, G, epoch)) break;
        // 5. the exact step (CTA 0)
        if (blockIdx.x == 0) {
            double *key = reinterpret_cast<double *>(pcd_smem);
            double *jmp = key + KCAP;
            int *kid = reinterpret_cast<int *>(jmp + KCAP);
            const int nk = *reinterpret_cast<volatile int *>(&st->nk);
            double t, kinkt;
            pcd_walk(v, lam, g1, g2, h0, R, nk, key, jmp, kid, red, t, kinkt);
            if (threadIdx.x == 0) {
                st->t = t;
                st->kinkt = kinkt;
                st->nk = 0;
            }
        }
        if (!pcd_barrier(st, G, epoch)) break;
        const double t = __ldcg(&st->t), kinkt = __ldcg(&st->kinkt);
        // 6. Delta += t P with the exact zeros; b += t (W P W); corrections (into vq)
        for (int64_t p = lo + threadIdx.x; p < hi; p += PT) {
            const double P = v.P[p];
            double cr = 0.0;
            v.dprev[p] = v.d[p];
            if (P != 0.0) {
                const double c = v.c[p], D0 = v.D[p], A = v.aval[p];
                double nd;
                bool special = false;
                if (kinkt >= 0.0 && c != 0.0 && -c / P == kinkt && sgnd(c) != sgnd(P)) {
                    nd = -A;  // lands on the kink: an exact zero
                    special = true;
                } else {
                    nd = D0 + t * P;
                }
                if (v.zt[p] && c != 0.0 && nd == D0) {
                    nd = -A;  // the zero snap
                    special = true;
                }
                v.D[p] = nd;
                if (special) cr = (nd - D0) - t * P;
            }
            v.corr[p] = cr;
            v.vq[v.qi[p]] = cr;
            v.vq[v.qj[p]] = cr;
            v.b[p] += t * __ldcg(v.wpw + p);
            if (cr != 0.0) corr_pending = true;
        }
        ++it;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->it = it;
        st->d0max = d0max;
        st->done = 1;
    }
}

constexpr size_t PCD_SMEM = (size_t)KCAP * (2 * sizeof(double) + sizeof(int));
static_assert(PCD_SMEM >= 4 * (size_t)SP_ROWS * (SP_COLS + 1) * sizeof(float) &&
                  PCD_SMEM >= 2 * (size_t)SP_ROWS * (SP_COLS + 1) * sizeof(double),
              "the SpMM tiles fit");
constexpr size_t PCD_DYN_MAX = PCD_SMEM;  // the dynamic shared memory of k_pcd_persist (the walk's)

OncePerDevice g_pcd_once[2];
int g_pcd_nsm[2][kMaxDevices], g_pcd_occ[2][kMaxDevices];

// The per-row and fixed part of the scratch: CSR row pointers, cursors and
// counts (n + 1 each), then, 16-byte aligned, the state, the partials (2 x 4
// per CTA, at most PCD_MAX_G CTAs) and the gathered kinks (KCAP times, jumps,
// pair indices).
size_t pcd_rows_bytes(int64_t n) {
    return (size_t)(n + 1) * 3 * sizeof(int) + 16 + sizeof(PcdState) + 8 * PCD_MAX_G * sizeof(double) +
           (size_t)KCAP * (2 * sizeof(double) + sizeof(int)) + 64;
}

cudaError_t pcd_ensure(Work &w, int64_t n, int64_t np, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (np > w.pcd_cap_np) {
        // 8 pair vectors of doubles (b, c, d, d_prev, P, W P W, corrections,
        // scratch), the SpMM's entry values (2 np doubles), the CSR columns
        // and pair indices (2 np ints each), each pair's two CSR positions
        // (np ints each), the zero flags (np bytes)
        const int64_t cap = std::max<int64_t>(np, 2 * w.pcd_cap_np);
        if (w.pcd_vec && (e = cudaFreeAsync(w.pcd_vec, st)) != cudaSuccess) return e;
        w.pcd_vec = nullptr;
        w.pcd_cap_np = 0;
        const size_t bytes = (size_t)cap * (10 * sizeof(double) + 6 * sizeof(int) + 1) + 256;
        if ((e = cudaMallocAsync((void **)&w.pcd_vec, bytes, st)) != cudaSuccess) return e;
        w.pcd_cap_np = cap;
    }
    if (n + 1 > w.pcd_cap_n) {
        if (w.pcd_rows && (e = cudaFreeAsync(w.pcd_rows, st)) != cudaSuccess) return e;
        w.pcd_rows = nullptr;
        w.pcd_cap_n = 0;
        if ((e = cudaMallocAsync((void **)&w.pcd_rows, pcd_rows_bytes(n), st)) != cudaSuccess) return e;
        w.pcd_cap_n = n + 1;
    }
    return cudaSuccess;
}

}  // namespace

// PCD-CG on the pair list (see the top of the file).  W, U (n x n, T), Vt
// (n x n, T, scratch); inva, g, aval: 1/a, G and A on the pairs (pair_prep);
// D on the pairs (in/out), U = Delta W on return.  D may be nonzero on entry
// (then b starts from (W Delta W) of it).  *iters_done (host, optional)
// receives the iterations taken; the call synchronises the stream.
// cudaErrorLaunchTimeout: a bounded grid-barrier wait expired.
template <typename T>
cudaError_t pcd_t(const T *W, int64_t n, double lam, const int32_t *pi, const int32_t *pj, int64_t np,
                  const double *inva, const double *g, const double *aval, int iters, int cg, double rtol,
                  double *D, T *U, T *Vt, bool d_nonzero, Work &w, cudaStream_t st, int *iters_done) {
    if (iters_done) *iters_done = 0;
    if (np <= 0) return cudaMemsetAsync(U, 0, (size_t)(n * n) * sizeof(T), st);
    if (iters <= 0) return cudaSuccess;
    if (np > 0x7fffffff / 2) return cudaErrorInvalidValue;
    const int which = sizeof(T) == 8 ? 1 : 0;
    int dev = 0;
    cudaError_t e = g_pcd_once[which].run(dev, [&](int d) {
        cudaError_t e2 = cudaFuncSetAttribute(k_pcd_persist<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)PCD_DYN_MAX);
        if (e2 != cudaSuccess) return e2;
        e2 = cudaDeviceGetAttribute(&g_pcd_nsm[which][d], cudaDevAttrMultiProcessorCount, d);
        if (e2 != cudaSuccess) return e2;
        e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_pcd_occ[which][d], k_pcd_persist<T>, PT, PCD_DYN_MAX);
        if (e2 != cudaSuccess) return e2;
        return g_pcd_occ[which][d] < 1 ? cudaErrorInvalidConfiguration : cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    e = pcd_ensure(w, n, np, st);
    if (e != cudaSuccess) return e;
    // carve the scratch
    double *base = reinterpret_cast<double *>(w.pcd_vec);
    PcdVec v;
    v.pi = pi;
    v.pj = pj;
    v.inva = inva;
    v.g = g;
    v.aval = aval;
    v.D = D;
    v.b = base;
    v.c = base + np;
    v.d = base + 2 * np;
    v.dprev = base + 3 * np;
    v.P = base + 4 * np;
    v.wpw = base + 5 * np;
    v.corr = base + 6 * np;
    v.tmp = base + 7 * np;
    v.vq = base + 8 * np;
    int *col = reinterpret_cast<int *>(base + 10 * np);
    int *pid = col + 2 * np;
    int *qi = pid + 2 * np, *qj = qi + np;
    v.qi = qi;
    v.qj = qj;
    v.zt = reinterpret_cast<uint8_t *>(qj + np);
    v.np = np;
    int *ptr = w.pcd_rows, *cursor = ptr + (n + 1), *cnt = cursor + (n + 1);
    PcdState *sd = reinterpret_cast<PcdState *>(
        (reinterpret_cast<uintptr_t>(cnt + (n + 1)) + 15) & ~uintptr_t(15));
    static_assert(sizeof(PcdState) % 8 == 0, "the state keeps the partials aligned");
    v.part = reinterpret_cast<double *>(sd + 1);
    v.kt = v.part + 8 * PCD_MAX_G;
    v.kj = v.kt + KCAP;
    v.kp = reinterpret_cast<int *>(v.kj + KCAP);
    // CSR of the pairs
    const unsigned gp = (unsigned)lmax(1, lmin((np + 255) / 256, 152 * 8));
    if ((e = cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(int), st)) != cudaSuccess) return e;
    k_csr_count<<<gp, 256, 0, st>>>(pi, pj, np, cnt);
    k_csr_scan<<<1, 1024, 0, st>>>(cnt, n, ptr, cursor);
    k_csr_fill<<<gp, 256, 0, st>>>(pi, pj, np, cursor, col, pid);
    k_csr_sort<<<(unsigned)lmax(1, lmin((n + 255) / 256, 152 * 8)), 256, 0, st>>>(ptr, n, col, pid);
    k_csr_pos<<<(unsigned)lmax(1, lmin((2 * np + 255) / 256, 152 * 8)), 256, 0, st>>>(ptr, n, col, pid, pi, pj, qi,
                                                                                     qj);
    counted(5);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sd, 0, sizeof(PcdState), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(v.P, 0, (size_t)np * sizeof(double), st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(v.b, g, (size_t)np * sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    const dim3 tgrid((unsigned)lmin(((n + SP_ROWS - 1) / SP_ROWS) * ((n + SP_COLS - 1) / SP_COLS), 152 * 8));
    if (d_nonzero) {  // b = G + (W Delta W) on the pairs
        k_pair_spmm<T, true><<<tgrid, 256, 0, st>>>(W, n, ptr, col, pid, D, Vt);
        k_pair_sddmm<T><<<(unsigned)lmax(1, lmin((np + 7) / 8, 152 * 16)), 256, 0, st>>>(W, Vt, n, pi, pj, np,
                                                                                         v.tmp);
        k_vec_add<<<gp, 256, 0, st>>>(v.b, v.tmp, np);
        counted(3);
    }
    // all iterations: one cooperative launch, one CTA per SM at most, and no
    // more than the SpMM tiles and the pairs can use (a small problem leaves
    // the other SMs to the work beside it)
    const int64_t tiles = ((n + SP_ROWS - 1) / SP_ROWS) * ((n + SP_COLS - 1) / SP_COLS);
    const int64_t want = lmax(tiles / 2, (np + 127) / 128);
    const int G = (int)lmax(1, lmin(lmin((int64_t)g_pcd_nsm[which][dev] * g_pcd_occ[which][dev], PCD_MAX_G), want));
    // rows per SpMM tile: halved (down to 8) while the grid's warp groups
    // outnumber the tiles (at n = 494, 32-row tiles gave 64 tiles to 600
    // groups, each tile a long chain of dependent row gathers)
    const int64_t tcols = (n + SP_COLS - 1) / SP_COLS;
    int sr = SP_ROWS;
    while (sr > 8 && ((n + sr - 1) / sr) * tcols < (int64_t)G * SPLIT_NH<T>) sr /= 2;
    v.sr = sr;
    void *args[] = {(void *)&W, (void *)&Vt, (void *)&n, (void *)&lam, (void *)&ptr, (void *)&col,
                    (void *)&pid, (void *)&v, (void *)&iters, (void *)&cg, (void *)&rtol, (void *)&sd};
    e = cudaLaunchCooperativeKernel((const void *)k_pcd_persist<T>, dim3(G), dim3(PT), args, PCD_SMEM, st);
    counted(1);
    if (e != cudaSuccess) return e;
    // U = Delta W
    k_pair_spmm<T, false><<<tgrid, 256, 0, st>>>(W, n, ptr, col, pid, D, U);
    counted(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    PcdState hs;
    if ((e = cudaMemcpyAsync(&hs, sd, sizeof(PcdState), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (iters_done) *iters_done = hs.it;
    return hs.err ? cudaErrorLaunchTimeout : cudaSuccess;
}

cudaError_t pcd(const double *W, int64_t n, double lam, const int32_t *pi, const int32_t *pj, int64_t np,
                const double *inva, const double *g, const double *aval, int iters, int cg, double rtol,
                double *D, double *U, double *Vt, bool d_nonzero, Work &w, cudaStream_t st, int *iters_done) {
    return pcd_t<double>(W, n, lam, pi, pj, np, inva, g, aval, iters, cg, rtol, D, U, Vt, d_nonzero, w, st,
                         iters_done);
}

cudaError_t pcd32(const float *W, int64_t n, double lam, const int32_t *pi, const int32_t *pj, int64_t np,
                  const double *inva, const double *g, const double *aval, int iters, int cg, double rtol,
                  double *D, float *U, float *Vt, bool d_nonzero, Work &w, cudaStream_t st, int *iters_done) {
    return pcd_t<float>(W, n, lam, pi, pj, np, inva, g, aval, iters, cg, rtol, D, U, Vt, d_nonzero, w, st,
                        iters_done);
}

}  // namespace glx
