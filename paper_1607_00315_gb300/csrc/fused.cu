// The batched solver: whole solves of many small problems in one persistent
// launch.
//
// Each CTA takes a lambda-path (a run of problems on the same S, each warm
// started from the previous solution: the continuation at the end of Section
// 2) from an atomic queue and runs every step of every ML-cycle of its
// problems itself (Algorithm 1 with nu = nu_c = 1 and the hierarchy of
// Section 7; the dense proximal-Newton relaxation of Sections 5.1-5.2):
//   factorisation A = L L^T (the positive-definiteness test and log det),
//   X = L^{-1} and W = X^T X = A^{-1}                     (eq. gradHes)
//   the free set and the relative KKT residual           (eq. active_set, Section 8)
//   the nested candidate sets of the next cycle          (Section 7)
//   the Newton direction by CD sweeps                    (eq. Quad_MLE_l1_prior, eq. 1d_l1)
//   the Armijo backtracking line search                  (Section 6.1.2)
// Every decision (the KKT stop, the level, the line-search acceptance, the next
// path) is taken on the device; the host launches once and reads the results.
// The arithmetic is FP64 throughout and the steps are taken in the order of
// the FP64 solver, so the iterates follow it up to the rounding of
// differently ordered sums.
//
// Layout: n <= GLASSO_FUSED_MAX_N = FUSED_THREADS, so one thread owns one column of a
// row.  Per CTA a workspace slot holds A, W, T (the factor), X (the inverse
// factor) and Ut (the transpose of U = Delta W of the sweep), n x n FP64 each,
// and the pair lists with the sweep's per-pair scalars (capacity n (n + 1) / 2).
#include <math.h>

#include "glasso_internal.h"

namespace glx {
namespace {

constexpr int FT = FUSED_THREADS;
constexpr int FW = FT / 32;
constexpr int PNB = 16;       // panel width of the factorisation and of the inverse
constexpr int PLD = PNB + 1;  // padded row of a staged panel
constexpr int MAX_LEVELS = 62;
constexpr int LS_TRIALS = 30;
constexpr double LS_SIGMA = 1e-4;

struct FShared {
    double red[2][FW];  // reduction partials (two buffers: the sweep alternates)
    double redm[FW];
    int wcnt[FW];       // per-warp counts of a compaction
    unsigned hist[256]; // radix-select histogram
    long long sizes[MAX_LEVELS + 2];
    long long lbc[4];   // broadcast integers
    double dbc[2];      // broadcast doubles
    int ibc;
    int fail;
    double cls[FUSED_CLASSES];  // device time per step class of the current solve (thread 0)
    unsigned long long tmark;
    double dg[PNB][PLD];  // a diagonal block of the factor
    double dx[PNB][PLD];  // its inverse
    double panel[GLASSO_FUSED_MAX_N * PLD];
};

__device__ __forceinline__ double sgnd(double x) { return (double)((x > 0.0) - (x < 0.0)); }
__device__ __forceinline__ double softd(double x, double t) {
    // soft shrinkage S_t(x) = sign(x) max(|x| - t, 0)
    const double m = fabs(x) - t;
    return m > 0.0 ? copysign(m, x) : 0.0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum over the CTA.  Every thread returns the same value: the warp partials
// are added in warp order by each thread.
__device__ double cta_sum(double v, FShared &sm) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm.red[0][threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < FW; ++k) s += sm.red[0][k];
    return s;
}

__device__ double cta_max(double v, FShared &sm) {
    v = warp_max(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm.redm[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < FW; ++k) s = fmax(s, sm.redm[k]);
    return s;
}

// Ordered compaction step: the position of this thread's flagged element among
// the flagged elements of the CTA (in thread order) and their total.
__device__ int cta_compact(bool f, int &total, FShared &sm) {
    const unsigned b = __ballot_sync(0xffffffffu, f);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm.wcnt[w] = __popc(b);
    __syncthreads();
    int off = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < FW; ++k) {
        const int c = sm.wcnt[k];
        off += k < w ? c : 0;
        tot += c;
    }
    total = tot;
    return off + __popc(b & ((1u << lane) - 1u));
}

__device__ __forceinline__ void tile_of(int idx, int &I, int &J) {
    // idx-th tile (I, J), J <= I, of a lower triangle enumerated row by row
    int i = (int)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > idx) --i;
    while ((i + 1) * (i + 2) / 2 <= idx) ++i;
    I = i;
    J = idx - i * (i + 1) / 2;
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Thread 0 charges the time since the last mark to step class c (each step
// ends at a CTA barrier, so thread 0's clock stands for the CTA's).
__device__ __forceinline__ void lap(FShared &sm, int c) {
    if (threadIdx.x == 0) {
        const unsigned long long now = globaltimer();
        sm.cls[c] += (double)(now - sm.tmark);
        sm.tmark = now;
    }
}

// T <- the lower triangle of A (the upper triangle of T is not written).
__device__ void copy_lower(const double *A, double *T, int n) {
    const int nn = n * n;
    for (int e = threadIdx.x; e < nn; e += FT) {
        const int r = e / n, c = e - r * n;
        if (c <= r) T[e] = A[e];
    }
}

// ---- a2: Cholesky of the lower triangle, in place -----------------------
// Right-looking by panels of PNB columns: warp 0 factors the diagonal block
// in shared memory, one thread per row solves the panel below it against the
// block, and the trailing lower triangle takes the panel's rank-PNB update in
// 4 x 4 register tiles.  Returns 0 with logdet = sum_i log d_i (d_i the
// pivots, so log det = sum log L_ii^2), or k + 1 when pivot k is not positive
// (the matrix is not positive definite; Section 6.1.2's test).
__device__ int cta_potrf(double *M, int n, double &logdet, FShared &sm) {
    const int t = threadIdx.x, lane = t & 31;
    double ldsum = 0.0;
    for (int kb = 0; kb < n; kb += PNB) {
        const int nb = min(PNB, n - kb);
        if (t < 32) {
            if (lane < nb)
                for (int c = 0; c <= lane; ++c) sm.dg[lane][c] = M[(size_t)(kb + lane) * n + kb + c];
            __syncwarp();
            int bad = 0;
            for (int c = 0; c < nb; ++c) {
                const double d = sm.dg[c][c];  // the same value in every lane
                if (!(d > 0.0) || !(d < INFINITY)) {
                    bad = kb + c + 1;
                    break;
                }
                const double l = sqrt(d);
                if (lane == 0) ldsum += log(d);
                __syncwarp();
                if (lane == c) sm.dg[c][c] = l;
                if (lane > c && lane < nb) sm.dg[lane][c] /= l;
                __syncwarp();
                if (lane > c && lane < nb) {
                    const double v = sm.dg[lane][c];
                    for (int cc = c + 1; cc <= lane; ++cc) sm.dg[lane][cc] -= v * sm.dg[cc][c];
                }
                __syncwarp();
            }
            if (lane == 0) sm.fail = bad;
            if (!bad && lane < nb)
                for (int c = 0; c <= lane; ++c) M[(size_t)(kb + lane) * n + kb + c] = sm.dg[lane][c];
        }
        __syncthreads();
        if (sm.fail) {
            const int f = sm.fail;
            __syncthreads();
            return f;
        }
        const int m = n - kb - nb;
        if (m > 0) {
            // panel: row r solves x L_kk^T = a
            for (int r = t; r < m; r += FT) {
                const size_t row = (size_t)(kb + nb + r) * n + kb;
                double x[PNB];
#pragma unroll
                for (int c = 0; c < PNB; ++c) x[c] = c < nb ? M[row + c] : 0.0;
#pragma unroll
                for (int c = 0; c < PNB; ++c) {
                    if (c < nb) {
                        double s = x[c];
#pragma unroll
                        for (int cc = 0; cc < c; ++cc) s -= x[cc] * sm.dg[c][cc];
                        x[c] = s / sm.dg[c][c];
                    }
                }
#pragma unroll
                for (int c = 0; c < PNB; ++c)
                    if (c < nb) {
                        M[row + c] = x[c];
                        sm.panel[r * PLD + c] = x[c];
                    }
            }
            __syncthreads();
            // trailing update of the lower triangle
            const int q = (m + 3) >> 2;
            const int ntile = q * (q + 1) / 2;
            for (int idx = t; idx < ntile; idx += FT) {
                int I, J;
                tile_of(idx, I, J);
                const int r0 = 4 * I, c0 = 4 * J;
                double acc[4][4];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int s = 0; s < 4; ++s) acc[r][s] = 0.0;
                for (int c = 0; c < nb; ++c) {
                    double a[4], b[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) a[r] = r0 + r < m ? sm.panel[(r0 + r) * PLD + c] : 0.0;
#pragma unroll
                    for (int s = 0; s < 4; ++s) b[s] = c0 + s < m ? sm.panel[(c0 + s) * PLD + c] : 0.0;
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int s = 0; s < 4; ++s) acc[r][s] = fma(a[r], b[s], acc[r][s]);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        const int row = r0 + r, col = c0 + s;
                        if (row < m && col <= row) M[(size_t)(kb + nb + row) * n + kb + nb + col] -= acc[r][s];
                    }
            }
        }
        __syncthreads();
    }
    if (t == 0) sm.dbc[0] = ldsum;
    __syncthreads();
    logdet = sm.dbc[0];
    __syncthreads();
    return 0;
}

// ---- a3: X = L^{-1} (zeros written above the diagonal) ------------------
// By block rows of PNB: warp 0 inverts the diagonal block (lane c forward-
// substitutes column c), then X_I,J<I = -X_II (L_I,<I X_<I,<I), one thread
// per column of the block row.
__device__ void cta_trtri(const double *L, double *X, int n, FShared &sm) {
    const int t = threadIdx.x, lane = t & 31;
    for (int kb = 0; kb < n; kb += PNB) {
        const int nb = min(PNB, n - kb);
        if (t < 32) {
            if (lane < nb)
                for (int c = 0; c <= lane; ++c) sm.dg[lane][c] = L[(size_t)(kb + lane) * n + kb + c];
            __syncwarp();
            if (lane < nb) {
                const int c = lane;
                for (int r = 0; r < c; ++r) sm.dx[r][c] = 0.0;
                sm.dx[c][c] = 1.0 / sm.dg[c][c];
                for (int r = c + 1; r < nb; ++r) {
                    double s = 0.0;
                    for (int k = c; k < r; ++k) s += sm.dg[r][k] * sm.dx[k][c];
                    sm.dx[r][c] = -s / sm.dg[r][r];
                }
            }
            __syncwarp();
            if (lane < nb)
                for (int c = 0; c < nb; ++c) X[(size_t)(kb + lane) * n + kb + c] = sm.dx[lane][c];
        }
        __syncthreads();
        for (int j = t; j < kb; j += FT) {
            double y[PNB];
#pragma unroll
            for (int r = 0; r < PNB; ++r) y[r] = 0.0;
            // X[k][j] = 0 for k < j (written as zeros), so a warp may start at
            // its first column
            const int k0 = j & ~31;
            for (int k = k0; k < kb; ++k) {
                const double xk = X[(size_t)k * n + j];
#pragma unroll
                for (int r = 0; r < PNB; ++r)
                    if (r < nb) y[r] = fma(L[(size_t)(kb + r) * n + k], xk, y[r]);
            }
#pragma unroll
            for (int r = 0; r < PNB; ++r)
                if (r < nb) {
                    double s = 0.0;
#pragma unroll
                    for (int r2 = 0; r2 <= r; ++r2) s = fma(sm.dx[r][r2], y[r2], s);
                    X[(size_t)(kb + r) * n + j] = -s;
                }
        }
        const int wide = n - kb - nb;  // zeros right of the block
        for (int e = t; e < nb * wide; e += FT) {
            const int r = e / wide, c = kb + nb + (e - r * wide);
            X[(size_t)(kb + r) * n + c] = 0.0;
        }
        __syncthreads();
    }
}

// W = X^T X, both triangles: W_ij = sum_{k >= max(i, j)} X_ki X_kj, 4 x 4
// register tiles over the lower triangle.
__device__ void cta_xtx(const double *X, double *W, int n) {
    const int q = (n + 3) >> 2;
    const int ntile = q * (q + 1) / 2;
    for (int idx = threadIdx.x; idx < ntile; idx += FT) {
        int I, J;
        tile_of(idx, I, J);
        const int i0 = 4 * I, j0 = 4 * J;
        double acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int s = 0; s < 4; ++s) acc[r][s] = 0.0;
        for (int k = i0; k < n; ++k) {
            const double *xr = X + (size_t)k * n;
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = i0 + r < n ? xr[i0 + r] : 0.0;
#pragma unroll
            for (int s = 0; s < 4; ++s) b[s] = j0 + s < n ? xr[j0 + s] : 0.0;
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int s = 0; s < 4; ++s) acc[r][s] = fma(a[r], b[s], acc[r][s]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int i = i0 + r, j = j0 + s;
                if (i < n && j <= i) {
                    W[(size_t)i * n + j] = acc[r][s];
                    W[(size_t)j * n + i] = acc[r][s];
                }
            }
    }
}

// tr(S A) and ||A||_1 over all n^2 entries (eq. MLE_l1_prior).
__device__ void cta_sums(const double *S, const double *A, int n, double &trSA, double &l1, FShared &sm) {
    double tr = 0.0, a1 = 0.0;
    const int nn = n * n;
    for (int e = threadIdx.x; e < nn; e += FT) {
        const double a = A[e];
        tr = fma(S[e], a, tr);
        a1 += fabs(a);
    }
    trSA = cta_sum(tr, sm);
    l1 = cta_sum(a1, sm);
}

// ---- a4: the free set over the upper triangle, in row-major order ---------
// mode 0: (i, j) is free when A_ij != 0 or |S_ij - W_ij| > lambda (eq.
// active_set), with the sums of the level-0 relaxation in out[]: the summed
// and the largest |minimum-norm subgradient| (eq. subgradient1; the relative
// KKT residual of Section 8 divides the sum by ||A||_1), tr(S A), ||A||_1 and
// nnz(A), each over both triangles.  mode 1: A_ij != 0 or |S_ij| > lambda (the
// initial free set, Section 7).  Writes the pairs and |S - W| on them; returns
// their count.  One row per pass (n <= FT).
__device__ int cta_scan_full(const double *S, const double *W, const double *A, int n, double lam,
                             int mode, int32_t *oi, int32_t *oj, double *oabs, double *out,
                             FShared &sm) {
    double ks = 0.0, km = 0.0, tr = 0.0, l1 = 0.0, nz = 0.0;
    int base = 0;
    for (int i = 0; i < n; ++i) {
        const int j = i + threadIdx.x;
        bool f = false;
        double g = 0.0;
        if (j < n) {
            const size_t e = (size_t)i * n + j;
            const double s = S[e], a = A[e];
            g = s - W[e];
            f = a != 0.0 || fabs(mode ? s : g) > lam;
            if (!mode) {
                const double wgt = j == i ? 1.0 : 2.0;
                const double r = a != 0.0 ? g + lam * sgnd(a) : softd(g, lam);
                ks += wgt * fabs(r);
                km = fmax(km, fabs(r));
                tr += wgt * s * a;
                l1 += wgt * fabs(a);
                nz += a != 0.0 ? wgt : 0.0;
            }
        }
        int tot;
        const int pos = cta_compact(f, tot, sm);
        if (f) {
            oi[base + pos] = i;
            oj[base + pos] = j;
            oabs[base + pos] = fabs(g);
        }
        base += tot;
    }
    if (!mode) {
        out[0] = cta_sum(ks, sm);
        out[1] = cta_max(km, sm);
        out[2] = cta_sum(tr, sm);
        out[3] = cta_sum(l1, sm);
        out[4] = cta_sum(nz, sm);
    }
    __syncthreads();
    return base;
}

// The free set restricted to the candidates of level `level` (the pairs of
// the fine list with tag >= level; eq. MLE_l1_prior_C), in list order.
__device__ int cta_scan_cand(const double *S, const double *W, const double *A, int n, double lam,
                             const int32_t *fi, const int32_t *fj, const uint8_t *tag, int level,
                             int nf, int32_t *oi, int32_t *oj, FShared &sm) {
    int base = 0;
    for (int p0 = 0; p0 < nf; p0 += FT) {
        const int p = p0 + threadIdx.x;
        bool f = false;
        int i = 0, j = 0;
        if (p < nf && tag[p] >= level) {
            i = fi[p];
            j = fj[p];
            const size_t e = (size_t)i * n + j;
            f = A[e] != 0.0 || fabs(S[e] - W[e]) > lam;
        }
        int tot;
        const int pos = cta_compact(f, tot, sm);
        if (f) {
            oi[base + pos] = i;
            oj[base + pos] = j;
        }
        base += tot;
    }
    __syncthreads();
    return base;
}

// ---- a5: the nested candidate sets of Section 7 --------------------------
// |C_1| = max(ceil(nf / 2), |supp|), |C_{l+1}| = max(ceil(|C_l| / 2), |supp|)
// until |C_L| = |supp|; C_l = supp + the |C_l| - |supp| non-support pairs of
// largest |G|, ties to the earlier pair.  tag[p] = the coarsest level holding
// pair p.  Per level the threshold key is found by an MSB-first radix select
// (8-bit digits of the |G| bits: for non-negative doubles the bit patterns
// order like the values), then one ordered pass takes the keys above it and
// the first of the keys equal to it.  Returns L.
__device__ int cta_hierarchy(const double *absg, const int32_t *fi, const int32_t *fj,
                             const double *A, int n, int nf, uint8_t *tag, uint8_t *sup,
                             FShared &sm) {
    const int t = threadIdx.x, lane = t & 31;
    double cnt = 0.0;
    for (int p = t; p < nf; p += FT) {
        const bool s = A[(size_t)fi[p] * n + fj[p]] != 0.0;
        sup[p] = s;
        cnt += s ? 1.0 : 0.0;
    }
    const long long ns = (long long)cta_sum(cnt, sm);
    if (t == 0) {
        long long s = ((long long)nf + 1) / 2;
        if (s < ns) s = ns;
        sm.sizes[1] = s;
        int L = 1;
        while (sm.sizes[L] > ns && L < MAX_LEVELS) {
            long long nxt = (sm.sizes[L] + 1) / 2;
            if (nxt < ns) nxt = ns;
            sm.sizes[++L] = nxt;
        }
        sm.ibc = L;
    }
    __syncthreads();
    const int L = sm.ibc;
    for (int p = t; p < nf; p += FT) tag[p] = sup[p] ? (uint8_t)L : (uint8_t)0;
    __syncthreads();
    for (int l = 1; l <= L; ++l) {
        const long long r = sm.sizes[l] - ns;  // non-support pairs in C_l
        if (r <= 0) break;                     // the sizes only decrease
        unsigned long long prefix = 0, mask = 0;
        long long rem = r, gt = 0;
        for (int shift = 56; shift >= 0; shift -= 8) {
            for (int b = t; b < 256; b += FT) sm.hist[b] = 0u;
            __syncthreads();
            for (int p0 = 0; p0 < nf; p0 += FT) {
                const int p = p0 + t;
                int bin = -1;
                if (p < nf && !sup[p]) {
                    const unsigned long long k = (unsigned long long)__double_as_longlong(absg[p]);
                    if ((k & mask) == prefix) bin = (int)((k >> shift) & 255u);
                }
                const unsigned peers = __match_any_sync(0xffffffffu, bin);
                if (bin >= 0 && lane == __ffs(peers) - 1) atomicAdd(&sm.hist[bin], (unsigned)__popc(peers));
            }
            __syncthreads();
            if (t == 0) {
                long long cum = 0;
                int b = 255;
                for (; b > 0; --b) {
                    if (cum + (long long)sm.hist[b] >= rem) break;
                    cum += sm.hist[b];
                }
                sm.lbc[0] = b;
                sm.lbc[1] = rem - cum;
                sm.lbc[2] = gt + cum;
            }
            __syncthreads();
            const int b = (int)sm.lbc[0];
            rem = sm.lbc[1];
            gt = sm.lbc[2];
            prefix |= (unsigned long long)b << shift;
            mask |= 255ull << shift;
            __syncthreads();
        }
        // key K = prefix: gt keys lie above it; the first `rem` equal keys join
        const unsigned long long K = prefix;
        long long eqbase = 0;
        for (int p0 = 0; p0 < nf; p0 += FT) {
            const int p = p0 + t;
            bool eq = false, in = false;
            if (p < nf && !sup[p]) {
                const unsigned long long k = (unsigned long long)__double_as_longlong(absg[p]);
                in = k > K;
                eq = k == K;
            }
            int tot;
            const int pos = cta_compact(eq, tot, sm);
            if (eq && eqbase + pos < rem) in = true;
            if (in) tag[p] = (uint8_t)l;
            eqbase += tot;
        }
        __syncthreads();
    }
    return L;
}

// ---- a6: CD sweeps on the Newton LASSO (eq. Quad_MLE_l1_prior) -------------
// For pair p = (i, j) in list order: a = W_ij^2 + W_ii W_jj (W_ii^2 on the
// diagonal), b = G_ij + (W Delta W)_ij, c = A_ij + Delta_ij, the 1-D minimiser
// mu = -c + S_{lambda/a}(c - b/a) (eq. 1d_l1); a zero of the shrinkage is
// written exactly (Delta_ij = -A_ij).  U = Delta W is kept as Ut = U^T so that
// (W Delta W)_ij = W_i,: . Ut_j,: reads two rows; the update adds mu W_j,: to
// column i of Ut and mu W_i,: to column j.
// The chain runs on CDW warps, one per SM sub-partition (FP64 issues at a
// small fraction of the FP32 rate, so every FP64 instruction of the serial
// chain counts): lane k of the group owns entries k, k + CDT, ... of a row;
// each warp adds the group's partial dots and computes mu itself, so one
// named barrier orders the partials and one the row updates.
constexpr int CDW = 4;
constexpr int CDT = CDW * 32;
constexpr int CDE = (GLASSO_FUSED_MAX_N + CDT - 1) / CDT;

__device__ __forceinline__ void cd_bar() { asm volatile("bar.sync 1, %0;" ::"n"(CDT) : "memory"); }

// The sweep's per-pair scalars: g = S_ij - W_ij, 1/a, lambda/a, A_ij.
__device__ void cta_pair_prep(const double *S, const double *W, const double *A, int n, double lam,
                              const int32_t *qi, const int32_t *qj, int np, double *pg, double *pinva,
                              double *plia, double *pa) {
    for (int p = threadIdx.x; p < np; p += FT) {
        const int i = qi[p], j = qj[p];
        const size_t ei = (size_t)i * n, ej = (size_t)j * n;
        const double wij = W[ei + j];
        const double a = i == j ? wij * wij : wij * wij + W[ei + i] * W[ej + j];
        const double inva = 1.0 / a;
        pg[p] = S[ei + j] - wij;
        pinva[p] = inva;
        plia[p] = lam * inva;
        pa[p] = A[ei + j];
    }
    __syncthreads();
}

// Returns the number of rows of U updated (the same in every thread).
__device__ long long cta_cd(const double *W, int n, const int32_t *qi, const int32_t *qj, int np,
                            int nsweeps, const double *pg, const double *pinva, const double *plia,
                            const double *pa, double *D, double *Ut, FShared &sm) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    long long rows = 0;
    if (w < CDW) {
        int par = 0;
        for (int sw = 0; sw < nsweeps; ++sw) {
            for (int p = 0; p < np; ++p) {
                const int i = qi[p], j = qj[p];
                const size_t ei = (size_t)i * n, ej = (size_t)j * n;
                // the pair's scalars are read before the barrier (D[p] is written after it)
                const double g = pg[p], inva = pinva[p], lia = plia[p], aij = pa[p], dp = D[p];
                double wi[CDE], wj[CDE], prod = 0.0;
#pragma unroll
                for (int q = 0; q < CDE; ++q) {
                    const int k = t + q * CDT;
                    wi[q] = 0.0;
                    wj[q] = 0.0;
                    if (k < n) {
                        wi[q] = W[ei + k];
                        wj[q] = W[ej + k];
                        prod = fma(wi[q], Ut[ej + k], prod);
                    }
                }
                prod = warp_sum(prod);
                if (lane == 0) sm.red[par][w] = prod;
                cd_bar();
                double wdw = sm.red[par][0];
#pragma unroll
                for (int k = 1; k < CDW; ++k) wdw += sm.red[par][k];
                par ^= 1;
                const double b = g + wdw, c = aij + dp;
                const double z = softd(c - b * inva, lia);
                double mu = -c + z;
                if (mu != 0.0) {
                    double nd;
                    if (z == 0.0) {
                        mu = -aij - dp;
                        nd = -aij;
                    } else {
                        nd = dp + mu;
                    }
                    if (t == 0) D[p] = nd;
#pragma unroll
                    for (int q = 0; q < CDE; ++q) {
                        const int k = t + q * CDT;
                        if (k < n) {
                            Ut[(size_t)k * n + i] += mu * wj[q];
                            if (i != j) Ut[(size_t)k * n + j] += mu * wi[q];
                        }
                    }
                    rows += i != j ? 2 : 1;
                    cd_bar();
                }
            }
        }
    }
    __syncthreads();
    if (t == 0) sm.lbc[3] = rows;
    __syncthreads();
    rows = sm.lbc[3];
    __syncthreads();
    return rows;
}

// ---- a7: Armijo backtracking (Section 6.1.2) -------------------------------
// delta = tr(G Delta) + lambda (||A + Delta||_1 - ||A||_1); trial alpha = 1,
// 1/2, ...: T = A + alpha Delta must factor (positive definite) and satisfy
// F(T) <= F(A) + sigma alpha delta + eps_F, eps_F = 1e-12 max(|F(A)|, n) (the
// FP64 resolution of the objective).  On success A <- T, the objective's
// parts are updated and T holds the factor of the new A.
__device__ int cta_line_search(const double *S, const double *W, double *A, double *T, int n,
                               double lam, const int32_t *qi, const int32_t *qj, int np,
                               const double *D, double &F, double &logdet, double &trSA,
                               double &l1, int &trials, FShared &sm) {
    double dl = 0.0, tsd = 0.0;
    for (int p = threadIdx.x; p < np; p += FT) {
        const int i = qi[p], j = qj[p];
        const size_t e = (size_t)i * n + j;
        const double wgt = i == j ? 1.0 : 2.0, a = A[e], d = D[p];
        dl += wgt * ((S[e] - W[e]) * d + lam * (fabs(a + d) - fabs(a)));
        tsd += wgt * S[e] * d;
    }
    const double delta = cta_sum(dl, sm);
    const double trSD = cta_sum(tsd, sm);
    const double epsF = 1e-12 * fmax(fabs(F), (double)n);
    double alpha = 1.0;
    for (int tr = 0; tr < LS_TRIALS; ++tr) {
        copy_lower(A, T, n);
        __syncthreads();
        double d1 = 0.0;
        for (int p = threadIdx.x; p < np; p += FT) {
            const int i = qi[p], j = qj[p];
            const double wgt = i == j ? 1.0 : 2.0, a = A[(size_t)i * n + j];
            const double v = a + alpha * D[p];
            T[(size_t)j * n + i] = v;
            d1 += wgt * (fabs(v) - fabs(a));
        }
        const double dl1 = cta_sum(d1, sm);
        double ld = 0.0;
        const int info = cta_potrf(T, n, ld, sm);
        trials = tr + 1;
        if (info == 0) {
            const double Ft = -ld + (trSA + alpha * trSD) + lam * (l1 + dl1);
            if (Ft <= F + LS_SIGMA * alpha * delta + epsF) {
                for (int p = threadIdx.x; p < np; p += FT) {
                    const int i = qi[p], j = qj[p];
                    const double v = A[(size_t)i * n + j] + alpha * D[p];
                    A[(size_t)i * n + j] = v;
                    A[(size_t)j * n + i] = v;
                }
                __syncthreads();
                F = Ft;
                logdet = ld;
                trSA += alpha * trSD;
                l1 += dl1;
                return GLASSO_OK;
            }
        }
        alpha *= 0.5;
    }
    return GLASSO_ELINESEARCH;
}

struct FSlot {
    double *A, *W, *T, *X, *Ut, *fabsg, *D, *pg, *pinva, *plia, *pa;
    int32_t *fi, *fj, *pi, *pj;
    uint8_t *ftag, *fsup;
};

__device__ __forceinline__ size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

__device__ FSlot carve(char *base, int nmax) {
    const size_t nn = (size_t)nmax * nmax, P = (size_t)nmax * (nmax + 1) / 2;
    FSlot s;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char *p = base + o;
        o += align256(bytes);
        return p;
    };
    s.A = (double *)take(nn * 8);
    s.W = (double *)take(nn * 8);
    s.T = (double *)take(nn * 8);
    s.X = (double *)take(nn * 8);
    s.Ut = (double *)take(nn * 8);
    s.fabsg = (double *)take(P * 8);
    s.D = (double *)take(P * 8);
    s.pg = (double *)take(P * 8);
    s.pinva = (double *)take(P * 8);
    s.plia = (double *)take(P * 8);
    s.pa = (double *)take(P * 8);
    s.fi = (int32_t *)take(P * 4);
    s.fj = (int32_t *)take(P * 4);
    s.pi = (int32_t *)take(P * 4);
    s.pj = (int32_t *)take(P * 4);
    s.ftag = (uint8_t *)take(P);
    s.fsup = (uint8_t *)take(P);
    return s;
}

// ---- a8: one solve (the ML-cycle) -------------------------------------------
// warm: the slot's A holds the previous problem's solution (the next lambda of
// a path).  The steps and their order are those of the FP64 solver: the
// initial iterate diag(1 / (S_ii + lambda)) (or the warm start), the initial
// free set {|S_ij| > lambda} + supp(A) with |G| on it; per cycle k the
// hierarchy of the last fine free set, then for l = L .. 0 the relaxation on
// C_l (at l = 0 the full free set, the KKT stop), nsweeps = min(1 + k / 3, 10)
// CD sweeps from Delta = 0 and the line search.  The factor of the accepted
// trial is the factor of the next iterate, so each relaxation factors once
// per trial and inverts once.
__device__ void fused_solve(const FusedProblem &P, FusedResult &R, const FSlot &ws, bool warm,
                            FShared &sm) {
    const int t = threadIdx.x;
    const int n = P.n;
    const double lam = P.lambda;
    const double *S = P.S;
    const int nn = n * n;
    const unsigned long long t0 = globaltimer();
    if (t == 0) {
        for (int c = 0; c < FUSED_CLASSES; ++c) sm.cls[c] = 0.0;
        sm.tmark = t0;
    }
    int status = GLASSO_EMAXITER, cycles = 0, relax = 0, lstrials = 0;
    long long sweeps = 0;
    double F = 0.0, logdet = 0.0, relkkt = INFINITY, maxkkt = INFINITY, trSA = 0.0, l1 = 0.0;
    double nnz = 0.0, max_nnz = 0.0;
    const double n3 = (double)n * n * n;
    double flops = 0.0;  // n^3/3 per factorisation, 2n^3/3 per inverse, the sweeps' 2n per dot and row
    bool chol_ok = false, W_ok = false, fresh = false;
    int nf = 0;
    double o5[5];

    // initial iterate
    if (P.A0) {
        for (int e = t; e < nn; e += FT) ws.A[e] = P.A0[e];
    } else if (!warm) {
        double bad = 0.0;
        for (int e = t; e < nn; e += FT) {
            const int r = e / n, c = e - r * n;
            double v = 0.0;
            if (r == c) {
                const double d = S[e] + lam;
                if (!(d > 0.0)) bad = 1.0;
                v = 1.0 / d;
            }
            ws.A[e] = v;
        }
        if (cta_sum(bad, sm) != 0.0) {
            status = GLASSO_ENOTPD;
            goto out;
        }
    }
    __syncthreads();
    copy_lower(ws.A, ws.T, n);
    __syncthreads();
    flops += n3 / 3.0;
    if (cta_potrf(ws.T, n, logdet, sm) != 0) {
        status = GLASSO_ENOTPD;
        goto out;
    }
    lap(sm, 0);
    chol_ok = true;
    cta_trtri(ws.T, ws.X, n, sm);
    cta_xtx(ws.X, ws.W, n);
    __syncthreads();
    lap(sm, 1);
    flops += 2.0 * n3 / 3.0;
    W_ok = true;
    nf = cta_scan_full(S, ws.W, ws.A, n, lam, 1, ws.fi, ws.fj, ws.fabsg, o5, sm);
    lap(sm, 2);

    for (int k = 0; k < P.max_cycles; ++k) {
        cycles = k + 1;
        const int nsweeps = min(1 + k / 3, 10);
        int Lv = cta_hierarchy(ws.fabsg, ws.fi, ws.fj, ws.A, n, nf, ws.ftag, ws.fsup, sm);
        lap(sm, 2);
        if (P.one_level) Lv = 0;
        for (int l = Lv; l >= 0; --l) {
            fresh = false;
            if (!chol_ok) {
                copy_lower(ws.A, ws.T, n);
                __syncthreads();
                flops += n3 / 3.0;
                if (cta_potrf(ws.T, n, logdet, sm) != 0) {
                    status = GLASSO_ENOTPD;
                    goto out;
                }
                lap(sm, 0);
                chol_ok = true;
            }
            if (!W_ok) {
                cta_trtri(ws.T, ws.X, n, sm);
                cta_xtx(ws.X, ws.W, n);
                __syncthreads();
                flops += 2.0 * n3 / 3.0;
                lap(sm, 1);
                W_ok = true;
            }
            int np;
            const int32_t *qi, *qj;
            if (l == 0) {
                np = cta_scan_full(S, ws.W, ws.A, n, lam, 0, ws.fi, ws.fj, ws.fabsg, o5, sm);
                nf = np;
                relkkt = o5[0] / o5[3];
                maxkkt = o5[1];
                trSA = o5[2];
                l1 = o5[3];
                nnz = o5[4];
                max_nnz = fmax(max_nnz, nnz);
                F = -logdet + trSA + lam * l1;
                qi = ws.fi;
                qj = ws.fj;
                fresh = true;
                lap(sm, 2);
                if (relkkt <= P.tol) {
                    status = GLASSO_OK;
                    goto out;
                }
            } else {
                cta_sums(S, ws.A, n, trSA, l1, sm);
                F = -logdet + trSA + lam * l1;
                np = cta_scan_cand(S, ws.W, ws.A, n, lam, ws.fi, ws.fj, ws.ftag, l, nf, ws.pi, ws.pj, sm);
                qi = ws.pi;
                qj = ws.pj;
                lap(sm, 2);
            }
            // Newton direction from Delta = 0
            for (int e = t; e < nn; e += FT) ws.Ut[e] = 0.0;
            for (int p = t; p < np; p += FT) ws.D[p] = 0.0;
            __syncthreads();
            cta_pair_prep(S, ws.W, ws.A, n, lam, qi, qj, np, ws.pg, ws.pinva, ws.plia, ws.pa);
            const long long rows =
                cta_cd(ws.W, n, qi, qj, np, nsweeps, ws.pg, ws.pinva, ws.plia, ws.pa, ws.D, ws.Ut, sm);
            sweeps += nsweeps;
            flops += 2.0 * n * ((double)np * nsweeps + (double)rows);
            lap(sm, 3);
            double mv = 0.0;
            for (int p = t; p < np; p += FT) mv += ws.D[p] != 0.0 ? 1.0 : 0.0;
            if (cta_sum(mv, sm) != 0.0) {
                int tr = 0;
                const int rc = cta_line_search(S, ws.W, ws.A, ws.T, n, lam, qi, qj, np, ws.D, F, logdet,
                                               trSA, l1, tr, sm);
                lstrials += tr;
                flops += tr * n3 / 3.0;
                lap(sm, 4);
                if (rc != GLASSO_OK) {
                    chol_ok = false;  // T holds a rejected trial
                    status = rc;
                    goto out;
                }
                W_ok = false;  // T holds the factor of the new A
                fresh = false;
            }
            ++relax;
        }
    }
out:
    if (!fresh && (status == GLASSO_OK || status == GLASSO_EMAXITER || status == GLASSO_ELINESEARCH)) {
        // final evaluation at A: factor, W, objective and KKT residual
        bool ok = true;
        if (!chol_ok) {
            copy_lower(ws.A, ws.T, n);
            __syncthreads();
            flops += n3 / 3.0;
            ok = cta_potrf(ws.T, n, logdet, sm) == 0;
        }
        if (ok) {
            if (!W_ok) {
                cta_trtri(ws.T, ws.X, n, sm);
                cta_xtx(ws.X, ws.W, n);
                __syncthreads();
                flops += 2.0 * n3 / 3.0;
            }
            cta_scan_full(S, ws.W, ws.A, n, lam, 0, ws.fi, ws.fj, ws.fabsg, o5, sm);
            relkkt = o5[0] / o5[3];
            maxkkt = o5[1];
            trSA = o5[2];
            l1 = o5[3];
            nnz = o5[4];
            F = -logdet + trSA + lam * l1;
        }
    }
    max_nnz = fmax(max_nnz, nnz);
    __syncthreads();
    for (int e = t; e < nn; e += FT) P.A_out[e] = ws.A[e];
    if (t == 0) {
        R.status = status;
        R.cycles = cycles;
        R.relaxations = relax;
        R.ls_trials = lstrials;
        R.objective = F;
        R.rel_kkt = relkkt;
        R.max_kkt = maxkkt;
        R.logdet = logdet;
        R.nnz = (long long)nnz;
        R.max_nnz = (long long)max_nnz;
        R.sweeps = sweeps;
        R.flops = flops;
        lap(sm, 2);  // the closing evaluation and the copy out
        for (int c = 0; c < FUSED_CLASSES; ++c) R.cls_ns[c] = sm.cls[c];
        R.t0 = t0;
        R.t1 = globaltimer();
    }
    __syncthreads();
}

// Persistent: each CTA pops paths (runs [first, end) of problems, the later
// ones warm started) from *next until none is left.  Paths are queued longest
// first by the host.
__global__ void __launch_bounds__(FT, 1)
    k_fused_paths(const FusedProblem *__restrict__ probs, FusedResult *__restrict__ res,
                  const int2 *__restrict__ paths, int npaths, int *next, char *arena,
                  size_t slot_bytes, int nmax) {
    extern __shared__ __align__(16) unsigned char fused_smem[];
    FShared &sm = *reinterpret_cast<FShared *>(fused_smem);
    const FSlot ws = carve(arena + (size_t)blockIdx.x * slot_bytes, nmax);
    for (int guard = 0; guard <= npaths; ++guard) {
        if (threadIdx.x == 0) sm.ibc = atomicAdd(next, 1);
        __syncthreads();
        const int c = sm.ibc;
        __syncthreads();
        if (c >= npaths) break;
        const int2 pa = paths[c];
        for (int k = pa.x; k < pa.y; ++k) fused_solve(probs[k], res[k], ws, k > pa.x, sm);
    }
}

}  // namespace

size_t fused_slot_bytes(int nmax) {
    auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t nn = (size_t)nmax * nmax, P = (size_t)nmax * (nmax + 1) / 2;
    return 5 * a(nn * 8) + 6 * a(P * 8) + 4 * a(P * 4) + 2 * a(P);
}

cudaError_t fused_paths(const FusedProblem *probs, FusedResult *res, const int2 *paths, int npaths,
                        int *next, char *arena, size_t slot_bytes, int nmax, int grid,
                        cudaStream_t st) {
    static OncePerDevice once;
    int dev = 0;
    cudaError_t e = once.run(dev, [](int) {
        return cudaFuncSetAttribute(k_fused_paths, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sizeof(FShared));
    });
    if (e != cudaSuccess) return e;
    if (npaths <= 0) return cudaSuccess;
    e = cudaMemsetAsync(next, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_fused_paths<<<grid, FT, sizeof(FShared), st>>>(probs, res, paths, npaths, next, arena, slot_bytes,
                                                    nmax);
    counted(1);
    return cudaGetLastError();
}

}  // namespace glx
