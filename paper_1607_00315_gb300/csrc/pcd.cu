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
// U is formed once at the end (SpMM of the final Delta).  The per-pair
// vector work runs as grid-wide passes whose last CTA reduces the partials
// and takes the scalar decisions (stop, CG coefficient, descent check, the
// step's bound); the kink walk runs in one CTA.  Every kernel reads a device
// flag and returns at once after the stopping rule fired, so the host
// launches iterations in chunks and synchronises once per chunk.  At the
// precision stop the coordinates whose own minimiser is zero take their
// exact zero (the final shrinkage).
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

constexpr int PT = 1024;          // threads of the one-CTA kernels
constexpr int KCAP = 4096;        // kinks sorted in shared memory
constexpr int SP_ROWS = 32;       // rows of V per SpMM CTA
constexpr int SP_COLS = 128;      // columns of V per SpMM CTA

struct PcdState {
    int done;        // the stopping rule fired: every later kernel returns at once
    int it;          // iterations completed
    int has_corr;    // exact zeros this iteration: b needs their correction
    int shrink;      // the precision stop fired: the final shrinkage is due
    int reset;       // the CG direction did not descend: back to the PCD direction
    int nk;          // kinks gathered in (0, R]
    unsigned arrive; // CTAs finished with the current pass (the last one resets it)
    int pad;
    double d0max;    // max |d| of the first iteration
    double beta, g1, g2, h0, R, t, kinkt;
};

__device__ __forceinline__ double sgnd(double x) { return (double)((x > 0.0) - (x < 0.0)); }
__device__ __forceinline__ double soft(double x, double th) {
    const double ax = fabs(x) - th;
    return ax > 0.0 ? copysign(ax, x) : 0.0;
}

// Block-wide sum over PT threads (every thread gets the result).
__device__ double block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double x = red[threadIdx.x];  // PT / 32 = 32 partials, in a fixed order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (threadIdx.x == 0) red[32] = x;
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
__global__ void __launch_bounds__(PT) k_csr_scan(const int *__restrict__ cnt, int64_t n,
                                                 int *__restrict__ ptr, int *__restrict__ cursor) {
    __shared__ int wsum[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int64_t per = (n + PT - 1) / PT, a = t * per, b = lmin(a + per, n);
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
    if (t == PT - 1) ptr[n] = off;
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

// ---------------------------------------------------------------- (W X W) on the pairs
// V = X W for the symmetric X given on the pairs (values x, CSR pattern):
// V_r = sum over the row's entries of x W_col.  A CTA forms a 32 x 128 block
// of V (rows strided over its 8 warps, columns over the lanes, every load a
// coalesced row segment of W) in shared memory and writes it out either
// transposed (TRANS: out = V^T, 32 consecutive elements per warp store) or
// as is.  Zero values are skipped.  `gate` (device, optional): return at once
// unless *gate != 0; `stop`: return at once when *stop != 0.
template <typename T, bool TRANS>
__global__ void __launch_bounds__(256) k_pair_spmm(const T *__restrict__ W, int64_t n,
                                                   const int *__restrict__ ptr, const int *__restrict__ col,
                                                   const int *__restrict__ pid, const double *__restrict__ x,
                                                   T *__restrict__ out, const int *gate, const int *stop) {
    if ((gate && *gate == 0) || (stop && *stop != 0)) return;
    __shared__ T tile[SP_ROWS][SP_COLS + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * SP_ROWS, k0 = (int64_t)blockIdx.y * SP_COLS;
    for (int rl = warp; rl < SP_ROWS; rl += 8) {
        const int64_t r = r0 + rl;
        T acc[SP_COLS / 32];
#pragma unroll
        for (int m = 0; m < SP_COLS / 32; ++m) acc[m] = T(0);
        if (r < n) {
            for (int q = ptr[r], qe = ptr[r + 1]; q < qe; ++q) {
                const T v = (T)x[pid[q]];
                if (v == T(0)) continue;
                const T *wr = W + (int64_t)col[q] * n + k0 + lane;
#pragma unroll
                for (int m = 0; m < SP_COLS / 32; ++m)
                    if (k0 + lane + 32 * m < n) acc[m] = fma(v, wr[32 * m], acc[m]);
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
    if (!TRANS) return;
    __syncthreads();
    for (int c = warp; c < SP_COLS; c += 8) {
        const int64_t k = k0 + c;
        if (k >= n) break;
        if (r0 + lane < n) out[k * n + r0 + lane] = tile[lane][c];
    }
}

// out_p = W_{i,:} . Vt_{j,:} (= (W X W)_ij for Vt = (X W)^T): one warp per
// pair, lanes over the row, sum in T.  Gated like k_pair_spmm.
template <typename T>
__global__ void __launch_bounds__(256) k_pair_sddmm(const T *__restrict__ W, const T *__restrict__ Vt,
                                                    int64_t n, const int32_t *__restrict__ pi,
                                                    const int32_t *__restrict__ pj, int64_t np,
                                                    double *__restrict__ out, const int *gate,
                                                    const int *stop) {
    if ((gate && *gate == 0) || (stop && *stop != 0)) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5), nw = (int64_t)gridDim.x * 8;
    for (int64_t p = w0; p < np; p += nw) {
        const T *a = W + (int64_t)pi[p] * n, *b = Vt + (int64_t)pj[p] * n;
        T s0 = T(0), s1 = T(0);
        int64_t k = lane;
        for (; k + 32 < n; k += 64) {
            s0 = fma(a[k], b[k], s0);
            s1 = fma(a[k + 32], b[k + 32], s1);
        }
        if (k < n) s0 = fma(a[k], b[k], s0);
        T s = s0 + s1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[p] = (double)s;
    }
}

// b += add on the pairs (the correction pass), gated.
__global__ void k_pcd_addb(double *__restrict__ b, const double *__restrict__ add, int64_t np,
                           const int *gate, const int *stop) {
    if ((gate && *gate == 0) || (stop && *stop != 0)) return;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x)
        b[p] += add[p];
}

// ---------------------------------------------------------------- one iteration, vector part
// The per-pair work of an iteration is a sequence of grid-wide passes over
// the pairs; each pass ends in per-CTA partial sums, and the last CTA to
// finish combines them in CTA order (deterministic) and takes the pass's
// scalar decision, which the next pass reads from the state.  Only the kink
// walk runs in one CTA, on the kinks gathered by the pass before it.
struct PcdVec {
    const int32_t *pi, *pj;
    const double *inva, *g, *aval;  // 1/a_p, G_p, A_p
    double *D, *b, *c, *d, *dprev, *P, *wpw, *corr;
    uint8_t *zt;
    int64_t np;
    double *part;      // 4 partials per CTA of a pass
    double *kt, *kj;   // gathered kinks: times and jumps (KCAP)
    int *kp;           //                  pair indices
};

constexpr int GT = 256;  // threads of a pass CTA

__device__ __forceinline__ double pair_w(const PcdVec &v, int64_t p) { return v.pi[p] == v.pj[p] ? 1.0 : 2.0; }

// Reduce NV per-thread values (slot k a max when bit k of maxmask is set, else
// a sum) over the grid; returns true in thread 0 of the last CTA to arrive,
// with the totals in out.  Partials are combined in CTA order.
template <int NV>
__device__ bool pass_reduce(double (&v)[NV], unsigned maxmask, double *part, unsigned *arrive,
                            double (&out)[NV]) {
    __shared__ double sred[NV][GT / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_xor_sync(0xffffffffu, x, o);
            x = (maxmask >> k) & 1u ? fmax(x, y) : x + y;
        }
        if (lane == 0) sred[k][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = sred[k][0];
            for (int w = 1; w < GT / 32; ++w) x = (maxmask >> k) & 1u ? fmax(x, sred[k][w]) : x + sred[k][w];
            part[blockIdx.x * NV + k] = x;
        }
        __threadfence();
        last = atomicAdd(arrive, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || wid != 0) return false;
    __threadfence();
    // warp 0 of the last CTA: lane l combines partials l, l + 32, ... in order
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const bool mx = (maxmask >> k) & 1u;
        double x = mx ? -INFINITY : 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) {
            const double y = __ldcg(part + b * NV + k);
            x = mx ? fmax(x, y) : x + y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_xor_sync(0xffffffffu, x, o);
            x = mx ? fmax(x, y) : x + y;
        }
        out[k] = x;
    }
    if (lane == 0) *arrive = 0u;
    return lane == 0;
}

// Pass 1: c, the PCD direction d, max|d| and the Polak-Ribiere sums; the
// last CTA applies the stopping rule and sets beta.
__global__ void __launch_bounds__(GT) k_pcd_dir(PcdVec v, double lam, int iters, int cg, double rtol,
                                                PcdState *st) {
    if (st->done) return;
    const int it = st->it;
    if (it >= iters) {
        if (blockIdx.x == 0 && threadIdx.x == 0) st->done = 1;
        return;
    }
    double r[3] = {0.0, 0.0, 0.0};  // max |d|, <d, d - d_prev>_w, <d_prev, d_prev>_w
    for (int64_t p = blockIdx.x * (int64_t)GT + threadIdx.x; p < v.np; p += (int64_t)gridDim.x * GT) {
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
    double o[3];
    if (!pass_reduce<3>(r, 1u, v.part, &st->arrive, o)) return;
    const double dmax = o[0];
    if (dmax == 0.0) {
        st->done = 1;
    } else if (it > 0 && rtol > 0.0 && dmax <= rtol * st->d0max) {
        st->done = 1;
        st->shrink = 1;  // the final shrinkage (k_pcd_shrink)
    } else {
        if (it == 0) st->d0max = dmax;
        st->beta = (cg && it > 0 && o[2] > 0.0) ? fmax(0.0, o[1] / o[2]) : 0.0;
    }
}

// At the precision stop: coordinates whose own minimiser is zero take their
// exact zero.  Runs after the stop (gated on `shrink` alone).
__global__ void __launch_bounds__(GT) k_pcd_shrink(PcdVec v, PcdState *st) {
    if (!st->shrink) return;
    for (int64_t p = blockIdx.x * (int64_t)GT + threadIdx.x; p < v.np; p += (int64_t)gridDim.x * GT) {
        const double c = v.c[p];
        if (c != 0.0 && c + v.d[p] == 0.0) v.D[p] = -v.aval[p];
    }
}

// Pass 2: P = d + beta P_prev, the zero flags, g1 = <b, P>_w and the slope h
// of the l1 term at 0+; the last CTA checks descent.
__global__ void __launch_bounds__(GT) k_pcd_dirP(PcdVec v, double lam, PcdState *st) {
    if (st->done) return;
    const double beta = st->beta;
    double r[2] = {0.0, 0.0};
    for (int64_t p = blockIdx.x * (int64_t)GT + threadIdx.x; p < v.np; p += (int64_t)gridDim.x * GT) {
        const double dp = v.d[p], c = v.c[p];
        const double P = dp + beta * v.P[p];  // P holds the previous direction (0 at the start)
        v.P[p] = P;
        v.zt[p] = c + dp == 0.0;  // the coordinate's own minimiser is zero
        const double w = pair_w(v, p);
        r[0] += w * v.b[p] * P;
        if (P != 0.0) r[1] += lam * w * P * (c != 0.0 ? sgnd(c) : sgnd(P));
    }
    double o[2];
    if (!pass_reduce<2>(r, 0u, v.part, &st->arrive, o)) return;
    st->g1 = o[0];
    st->reset = beta != 0.0 && o[0] + o[1] >= 0.0;  // not a descent direction
}

// Pass 2b (after a failed descent check): back to the PCD direction.
__global__ void __launch_bounds__(GT) k_pcd_reset(PcdVec v, PcdState *st) {
    if (st->done || !st->reset) return;
    double r[1] = {0.0};
    for (int64_t p = blockIdx.x * (int64_t)GT + threadIdx.x; p < v.np; p += (int64_t)gridDim.x * GT) {
        v.P[p] = v.d[p];
        r[0] += pair_w(v, p) * v.b[p] * v.d[p];
    }
    double o[1];
    if (!pass_reduce<1>(r, 0u, v.part, &st->arrive, o)) return;
    st->g1 = o[0];
    st->reset = 0;
}

// Pass 3 (after W P W): g2 = <P, W P W>_w and h(0+); the last CTA decides
// whether the step is zero and sets the bound R = -(g1 + h(0+)) / g2 of the
// minimiser.
__global__ void __launch_bounds__(GT) k_pcd_g2(PcdVec v, double lam, PcdState *st) {
    if (st->done) return;
    double r[2] = {0.0, 0.0};
    for (int64_t p = blockIdx.x * (int64_t)GT + threadIdx.x; p < v.np; p += (int64_t)gridDim.x * GT) {
        const double P = v.P[p];
        if (P == 0.0) continue;
        const double w = pair_w(v, p), c = v.c[p];
        r[0] += w * P * v.wpw[p];
        r[1] += lam * w * P * (c != 0.0 ? sgnd(c) : sgnd(P));
    }
    double o[2];
    if (!pass_reduce<2>(r, 0u, v.part, &st->arrive, o)) return;
    const double g2 = o[0], h0 = o[1], g1 = st->g1;
    st->g2 = g2;
    st->h0 = h0;
    st->nk = 0;
    if (!(g2 > 0.0) || g1 + h0 >= 0.0) {
        st->t = 0.0;
        st->done = 1;  // no descent along P: the oracle's zero step ends the iteration
    } else {
        st->R = -(g1 + h0) / g2;
    }
}

// Pass 4: gather the kinks t_p = -c_p / P_p in (0, R] (at most KCAP; the count
// beyond that sends the walk to its fallback).
__global__ void __launch_bounds__(GT) k_pcd_kinks(PcdVec v, double lam, PcdState *st) {
    if (st->done) return;
    const double R = st->R;
    for (int64_t p = blockIdx.x * (int64_t)GT + threadIdx.x; p < v.np; p += (int64_t)gridDim.x * GT) {
        const double P = v.P[p], c = v.c[p];
        if (P == 0.0 || c == 0.0 || sgnd(c) == sgnd(P)) continue;
        const double tk = -c / P;
        if (!(tk > 0.0 && tk <= R)) continue;
        const int s = atomicAdd(&st->nk, 1);
        if (s < KCAP) {
            v.kt[s] = tk;
            v.kj[s] = 2.0 * lam * pair_w(v, p) * fabs(P);
            v.kp[s] = (int)p;
        }
    }
}

// lambda sum_p w_p P_p sign(c_p + t P_p) (sign(P_p) where c_p + t P_p = 0) and
// the number of kinks in (L, R], over one thread's pairs (one-CTA kernel).
__device__ __forceinline__ void slope_and_kinks(const PcdVec &v, double lam, double t, double L, double R,
                                                double &h, double &cnt) {
    h = 0.0;
    cnt = 0.0;
    for (int64_t p = threadIdx.x; p < v.np; p += PT) {
        const double P = v.P[p];
        if (P == 0.0) continue;
        const double c = v.c[p], w = pair_w(v, p);
        const double x = c + t * P;
        h += lam * w * P * (x != 0.0 ? sgnd(x) : sgnd(P));
        if (c != 0.0 && sgnd(c) != sgnd(P)) {
            const double tk = -c / P;
            if (tk > L && tk <= R) cnt += 1.0;
        }
    }
}

// The exact step (one CTA; dynamic shared memory: KCAP keys, jumps and pair
// indices): sort the kinks of (L, R] and walk them in increasing order from
// h(L+).  L = 0 and the kinks gathered by k_pcd_kinks when they fit; else the
// interval is first halved (bit-pattern bisection on the sign of phi') over
// all pairs until its kinks fit, or until it holds a single kink value.
__global__ void __launch_bounds__(PT) k_pcd_walk(PcdVec v, double lam, PcdState *st) {
    extern __shared__ __align__(16) unsigned char pcd_smem[];
    double *key = reinterpret_cast<double *>(pcd_smem);
    double *jmp = key + KCAP;
    int *kid = reinterpret_cast<int *>(jmp + KCAP);
    __shared__ double red[33];
    __shared__ int nkink;
    if (st->done) return;
    const double g1 = st->g1, g2 = st->g2;
    double L = 0.0, HL = st->h0, R = st->R;
    bool group = false;  // (L, R] holds more than KCAP kinks, all at R
    int m = st->nk;
    if (m <= KCAP) {
        for (int s = threadIdx.x; s < m; s += PT) {
            key[s] = v.kt[s];
            jmp[s] = v.kj[s];
            kid[s] = v.kp[s];
        }
    } else {
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
        if (threadIdx.x == 0) nkink = 0;
        __syncthreads();
        double gjump = 0.0;
        for (int64_t p = threadIdx.x; p < v.np; p += PT) {
            const double P = v.P[p], c = v.c[p];
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
            if (threadIdx.x == 0) {
                double t = NAN, kinkt = -1.0, H = HL;
                const double ts = -(g1 + H) / g2;
                if (ts <= R) t = ts;
                else if (g1 + g2 * R + H + gjump >= 0.0) t = kinkt = R;
                else t = -(g1 + H + gjump) / g2;
                st->t = t;
                st->kinkt = kinkt;
            }
            return;
        }
        __syncthreads();
        m = min(nkink, KCAP);
    }
    __syncthreads();
    // bitonic sort of (key, pair index), padded to a power of two
    int m2 = 1;
    while (m2 < m) m2 <<= 1;
    for (int s = m + threadIdx.x; s < m2; s += PT) {
        key[s] = INFINITY;
        jmp[s] = 0.0;
        kid[s] = 0x7fffffff;
    }
    __syncthreads();
    for (int size = 2; size <= m2; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int s = threadIdx.x; s < m2; s += PT) {
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
    if (threadIdx.x != 0) return;
    // the walk, in increasing order from h(L+)
    double H = HL, t = NAN, kinkt = -1.0;
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
    st->t = t;
    st->kinkt = kinkt;
}

// Pass 5: Delta += t P with exact zeros at the kink and the zero snap, b +=
// t (W P W), d_prev = d, the corrections (increment - t P) of the exact
// zeros; the last CTA counts the iteration.
__global__ void __launch_bounds__(GT) k_pcd_update(PcdVec v, PcdState *st) {
    if (st->done) return;
    const double t = st->t, kinkt = st->kinkt;
    double r[1] = {0.0};
    for (int64_t p = blockIdx.x * (int64_t)GT + threadIdx.x; p < v.np; p += (int64_t)gridDim.x * GT) {
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
        v.b[p] += t * v.wpw[p];
        if (cr != 0.0) r[0] = 1.0;
    }
    double o[1];
    if (!pass_reduce<1>(r, 1u, v.part, &st->arrive, o)) return;
    st->has_corr = o[0] != 0.0;
    st->it += 1;
}

constexpr size_t PCD_SMEM = (size_t)KCAP * (2 * sizeof(double) + sizeof(int));
constexpr int PCD_CHUNK = 4;  // iterations launched between two looks at the stopping flag

OncePerDevice g_pcd_once;

template <typename T>
cudaError_t spmm_launch(const T *W, int64_t n, const int *ptr, const int *col, const int *pid,
                        const double *x, T *out, bool trans, const int *gate, const int *stop,
                        cudaStream_t st) {
    const dim3 grid((unsigned)((n + SP_ROWS - 1) / SP_ROWS), (unsigned)((n + SP_COLS - 1) / SP_COLS));
    if (trans)
        k_pair_spmm<T, true><<<grid, 256, 0, st>>>(W, n, ptr, col, pid, x, out, gate, stop);
    else
        k_pair_spmm<T, false><<<grid, 256, 0, st>>>(W, n, ptr, col, pid, x, out, gate, stop);
    counted(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t sddmm_launch(const T *W, const T *Vt, int64_t n, const int32_t *pi, const int32_t *pj,
                         int64_t np, double *out, const int *gate, const int *stop, cudaStream_t st) {
    const unsigned g = (unsigned)lmax(1, lmin((np + 7) / 8, 152 * 16));
    k_pair_sddmm<T><<<g, 256, 0, st>>>(W, Vt, n, pi, pj, np, out, gate, stop);
    counted(1);
    return cudaGetLastError();
}

// Scratch of the PCD solver, grown on demand (pair vectors for np pairs, the
// CSR of the pairs for n rows, the state).
// The per-row and fixed part: CSR row pointers, cursors and counts (n + 1 each),
// then, 16-byte aligned, the state, the pass partials (3 per CTA, at most 152
// CTAs) and the gathered kinks (KCAP times, jumps, pair indices).
size_t pcd_rows_bytes(int64_t n) {
    return (size_t)(n + 1) * 3 * sizeof(int) + 16 + sizeof(PcdState) + 3 * 152 * sizeof(double) +
           (size_t)KCAP * (2 * sizeof(double) + sizeof(int)) + 64;
}

cudaError_t pcd_ensure(Work &w, int64_t n, int64_t np, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (np > w.pcd_cap_np) {
        // 9 pair vectors of doubles (b, c, d, d_prev, P, W P W, corrections,
        // scratch, spare), the CSR columns and pair indices (2 np ints each),
        // the zero flags (np bytes)
        const int64_t cap = std::max<int64_t>(np, 2 * w.pcd_cap_np);
        if (w.pcd_vec && (e = cudaFreeAsync(w.pcd_vec, st)) != cudaSuccess) return e;
        w.pcd_vec = nullptr;
        w.pcd_cap_np = 0;
        const size_t bytes = (size_t)cap * (9 * sizeof(double) + 2 * 2 * sizeof(int) + 1) + 256;
        if ((e = cudaMallocAsync((void **)&w.pcd_vec, bytes, st)) != cudaSuccess) return e;
        w.pcd_cap_np = cap;
    }
    if (n + 1 > w.pcd_cap_n) {
        if (w.pcd_rows && (e = cudaFreeAsync(w.pcd_rows, st)) != cudaSuccess) return e;
        w.pcd_rows = nullptr;
        w.pcd_cap_n = 0;
        if ((e = cudaMallocAsync((void **)&w.pcd_rows, pcd_rows_bytes(n), st)) != cudaSuccess)
            return e;
        w.pcd_cap_n = n + 1;
    }
    return cudaSuccess;
}

}  // namespace

// PCD-CG on the pair list (see above).  W, U (n x n, T), Vt (n x n, T, scratch);
// inva, g, aval: 1/a, G and A on the pairs (pair_prep); D on the pairs (in/out),
// U = Delta W on return.  D may be nonzero on entry (then b starts from
// (W Delta W) of it).  *iters_done (host, optional) receives the iterations
// taken (the call then synchronises the stream).
template <typename T>
cudaError_t pcd_t(const T *W, int64_t n, double lam, const int32_t *pi, const int32_t *pj, int64_t np,
                  const double *inva, const double *g, const double *aval, int iters, int cg, double rtol,
                  double *D, T *U, T *Vt, bool d_nonzero, Work &w, cudaStream_t st, int *iters_done) {
    if (np <= 0 || iters <= 0) {
        if (iters_done) *iters_done = 0;
        return np <= 0 ? cudaMemsetAsync(U, 0, (size_t)(n * n) * sizeof(T), st) : cudaSuccess;
    }
    if (np > 0x7fffffff / 2) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = g_pcd_once.run(dev, [](int) {
        return cudaFuncSetAttribute(k_pcd_walk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PCD_SMEM);
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
    double *tmp = base + 7 * np;
    int *col = reinterpret_cast<int *>(base + 9 * np);
    int *pid = col + 2 * np;
    v.zt = reinterpret_cast<uint8_t *>(pid + 2 * np);
    v.np = np;
    int *ptr = w.pcd_rows, *cursor = ptr + (n + 1), *cnt = cursor + (n + 1);
    PcdState *sd = reinterpret_cast<PcdState *>(
        (reinterpret_cast<uintptr_t>(cnt + (n + 1)) + 15) & ~uintptr_t(15));
    v.part = reinterpret_cast<double *>(sd + 1);
    v.kt = v.part + 3 * 152;
    v.kj = v.kt + KCAP;
    v.kp = reinterpret_cast<int *>(v.kj + KCAP);
    static_assert(sizeof(PcdState) % 8 == 0, "state keeps the partials aligned");
    const unsigned gv = (unsigned)lmax(1, lmin((np + GT - 1) / GT, 152));
    // CSR of the pairs
    const unsigned gp = (unsigned)lmax(1, lmin((np + 255) / 256, 152 * 8));
    if ((e = cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(int), st)) != cudaSuccess) return e;
    k_csr_count<<<gp, 256, 0, st>>>(pi, pj, np, cnt);
    k_csr_scan<<<1, PT, 0, st>>>(cnt, n, ptr, cursor);
    k_csr_fill<<<gp, 256, 0, st>>>(pi, pj, np, cursor, col, pid);
    k_csr_sort<<<(unsigned)lmax(1, lmin((n + 255) / 256, 152 * 8)), 256, 0, st>>>(ptr, n, col, pid);
    counted(4);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sd, 0, sizeof(PcdState), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(v.P, 0, (size_t)np * sizeof(double), st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(v.b, g, (size_t)np * sizeof(double), cudaMemcpyDeviceToDevice, st)) !=
        cudaSuccess)
        return e;
    if (d_nonzero) {  // b = G + (W Delta W) on the pairs
        if ((e = spmm_launch<T>(W, n, ptr, col, pid, D, Vt, true, nullptr, nullptr, st)) != cudaSuccess) return e;
        if ((e = sddmm_launch<T>(W, Vt, n, pi, pj, np, tmp, nullptr, nullptr, st)) != cudaSuccess) return e;
        k_pcd_addb<<<gp, 256, 0, st>>>(v.b, tmp, np, nullptr, nullptr);
        counted(1);
    }
    PcdState hs{};
    for (int done_it = 0; done_it < iters;) {
        const int chunk = std::min(PCD_CHUNK, iters - done_it);
        for (int k = 0; k < chunk; ++k) {
            k_pcd_dir<<<gv, GT, 0, st>>>(v, lam, iters, cg, rtol, sd);
            k_pcd_shrink<<<gv, GT, 0, st>>>(v, sd);
            k_pcd_dirP<<<gv, GT, 0, st>>>(v, lam, sd);
            k_pcd_reset<<<gv, GT, 0, st>>>(v, sd);
            counted(4);
            if ((e = spmm_launch<T>(W, n, ptr, col, pid, v.P, Vt, true, nullptr, &sd->done, st)) != cudaSuccess)
                return e;
            if ((e = sddmm_launch<T>(W, Vt, n, pi, pj, np, v.wpw, nullptr, &sd->done, st)) != cudaSuccess)
                return e;
            k_pcd_g2<<<gv, GT, 0, st>>>(v, lam, sd);
            k_pcd_kinks<<<gv, GT, 0, st>>>(v, lam, sd);
            k_pcd_walk<<<1, PT, PCD_SMEM, st>>>(v, lam, sd);
            k_pcd_update<<<gv, GT, 0, st>>>(v, sd);
            counted(4);
            // the exact zeros' corrections (skipped unless has_corr)
            if ((e = spmm_launch<T>(W, n, ptr, col, pid, v.corr, Vt, true, &sd->has_corr, &sd->done, st)) !=
                cudaSuccess)
                return e;
            if ((e = sddmm_launch<T>(W, Vt, n, pi, pj, np, tmp, &sd->has_corr, &sd->done, st)) != cudaSuccess)
                return e;
            k_pcd_addb<<<gp, 256, 0, st>>>(v.b, tmp, np, &sd->has_corr, &sd->done);
            counted(1);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        done_it += chunk;
        if ((e = cudaMemcpyAsync(&hs, sd, sizeof(PcdState), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        if (hs.done) break;
    }
    if (iters_done) *iters_done = hs.it;
    // U = Delta W
    return spmm_launch<T>(W, n, ptr, col, pid, D, U, false, nullptr, nullptr, st);
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
