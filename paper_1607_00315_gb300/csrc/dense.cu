// Dense FP64 kernels of one relaxation: S = X^T X / m (eq. cov_estimate), the
// blocked right-looking Cholesky with PD test and log-det (Section 6.1.2 uses
// both in the line search), and W = A^{-1} = L^{-T} L^{-1} (eq. gradHes).
//
// GB300 note: FP64 runs at roughly 2 FMA/clock/SM on this part (about
// 1.1 TFLOP/s for the whole GPU), so every kernel here is bound by FP64
// issue, not by memory.  The design therefore maximises the number of
// independent 32 x 32 output tiles in flight (many small CTAs, several per
// SM) and keeps the serial panel work in shared memory.
#include <math.h>

#include "glasso_internal.h"
#include "leaf32.cuh"

namespace glx {
namespace {

constexpr int TPB = 256;  // threads of a tile CTA: 16 x 16, 2 x 2 outputs each

// acc += sum_{k in [k0, k1)} opA(i0 + i, k) * opB(k, j0 + j) for a 32 x 32 tile.
// opA(i, k) = TA ? A[k * lda + i] : A[i * lda + k]   (rows i < mrows)
// opB(k, j) = TB ? B[j * ldb + k] : B[k * ldb + j]   (cols j < ncols)
// Thread (ty, tx) owns rows {ty, ty + 16} and columns {tx, tx + 16}.
template <typename TIN, bool TA, bool TB, typename C = double>
__device__ __forceinline__ void tile_acc(C (&acc)[2][2], const TIN *__restrict__ A,
                                         int64_t lda, const TIN *__restrict__ B, int64_t ldb,
                                         int64_t i0, int64_t j0, int64_t k0, int64_t k1,
                                         int64_t mrows, int64_t ncols, C (*As)[NB + 1],
                                         C (*Bs)[NB + 1]) {
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    for (int64_t kc = k0; kc < k1; kc += NB) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int idx = tid + TPB * r;
            int i, k;
            if (TA) { i = idx & 31; k = idx >> 5; } else { k = idx & 31; i = idx >> 5; }
            int64_t gi = i0 + i, gk = kc + k;
            C v = 0;
            if (gi < mrows && gk < k1) v = (C)(TA ? A[gk * lda + gi] : A[gi * lda + gk]);
            As[k][i] = v;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int idx = tid + TPB * r;
            int j, k;
            if (TB) { k = idx & 31; j = idx >> 5; } else { j = idx & 31; k = idx >> 5; }
            int64_t gj = j0 + j, gk = kc + k;
            C v = 0;
            if (gj < ncols && gk < k1) v = (C)(TB ? B[gj * ldb + gk] : B[gk * ldb + gj]);
            Bs[k][j] = v;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < NB; ++k) {
            C a0 = As[k][ty], a1 = As[k][ty + 16];
            C b0 = Bs[k][tx], b1 = Bs[k][tx + 16];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
}

// Linear index over the lower-triangular tile grid (J <= I) -> (I, J).
__device__ __forceinline__ void tri_index(int64_t t, int64_t &I, int64_t &J) {
    int64_t i = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > t) --i;
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    I = i;
    J = t - i * (i + 1) / 2;
}

// ---------------------------------------------------------------- a1: S
template <typename TIN>
__global__ void k_stage_x(const TIN *__restrict__ X, int64_t m, int64_t n,
                          const double *__restrict__ mu, double *__restrict__ Xd) {
    int64_t total = m * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        double v = (double)X[t];
        if (mu) v -= mu[t % n];
        Xd[t] = v;
    }
}

template <typename TIN>
__global__ void k_colmean(const TIN *__restrict__ X, int64_t m, int64_t n, double *__restrict__ mu) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int64_t k = 0; k < m; ++k) s += (double)X[k * n + i];
    mu[i] = s / (double)m;
}

// S_IJ = sum_k X[k, I]^T X[k, J] / m on lower tiles, mirrored.
__global__ void __launch_bounds__(TPB) k_syrk_S(const double *__restrict__ X, int64_t m, int64_t n,
                                                double *__restrict__ S) {
    __shared__ double As[NB][NB + 1], Bs[NB][NB + 1];
    int64_t I, J;
    tri_index(blockIdx.x, I, J);
    double acc[2][2] = {{0, 0}, {0, 0}};
    tile_acc<double, true, false>(acc, X, n, X, n, I * NB, J * NB, 0, m, n, n, As, Bs);
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            int64_t i = I * NB + ty + 16 * a, j = J * NB + tx + 16 * b;
            if (i < n && j < n) {
                double v = acc[a][b] / (double)m;
                S[i * n + j] = v;
                S[j * n + i] = v;
            }
        }
}

// ---------------------------------------------------------------- a2: Cholesky
// Blocked right-looking factorisation with 32-wide panels.  The serial part
// of each step, factoring the 32 x 32 diagonal block and inverting its
// factor, is done by one warp in registers inside the trailing-update launch
// of the previous step (by the CTA that produces that block, which is
// scheduled first), so the panel itself is a parallel GEMM with the inverse:
//   step k:  L_ik = A_ik X_kk^T  (X_kk = L_kk^{-1})       k_potrf_panel
//            A_IJ -= L_Ik L_Jk^T, and factor block k+1   k_potrf_trail
// X_kk alternates between two 32 x 32 slots of `xd`.

// 1/sqrt(d) by Newton's iteration r <- r (3 - d r^2) / 2 from a
// single-precision seed (two steps reach full double precision); plain
// sqrt/division outside the single-precision range.
__device__ __forceinline__ double rsqrt_newton(double d) {
    if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
    double r = (double)rsqrtf((float)d);
    r = r * fma(-0.5 * d * r, r, 1.5);
    r = r * fma(-0.5 * d * r, r, 1.5);
    return r;
}

__device__ __forceinline__ float rsqrt_newton(float d) { return leaf::rsqrt_f32(d); }

// One warp factors the kw x kw lower block B (shared, row-major, padded) in
// place and writes Xs = L^{-1}, in the arithmetic of T.  (On this GPU one
// warp issues FP64 at a small fraction of its FP32 rate, so the FP32
// factorisation keeps its diagonal blocks in FP32.)  ldiag (global, optional)
// receives the diagonal of L as FP64 for the log-det.  Returns 0 or the
// failing pivot + 1 (same in every lane).  Lane i keeps row i in registers.
template <typename T>
__device__ int warp_chol_inv32(T (*B)[NB + 1], T (*Xs)[NB + 1], int kw, double *ldiag) {
    const int lane = threadIdx.x & 31;
    T a[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) a[c] = (lane < kw && c <= lane) ? B[lane][c] : (T)0;
    T rdiag = 0, lii = 0;
    int fail = 0;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (j < kw && !fail) {
            const T d = __shfl_sync(0xffffffffu, a[j], j);
            if (!(d > (T)0)) {
                fail = j + 1;
            } else {
                const T r = rsqrt_newton(d);
                if (lane == j) { a[j] = d * r; rdiag = r; lii = a[j]; }
                if (lane > j) a[j] *= r;
#pragma unroll
                for (int k = j + 1; k < NB; ++k) {
                    const T lkj = __shfl_sync(0xffffffffu, a[j], k);
                    if (lane >= k) a[k] = fma(-a[j], lkj, a[k]);
                }
            }
        }
    }
    if (fail) return fail;
    if (ldiag && lane < kw) ldiag[lane] = (double)lii;
    // keep the factor in shared memory (as T) and in FP64 for the inverse
#pragma unroll
    for (int c = 0; c < NB; ++c) B[lane][c] = a[c];
    __syncwarp();
    // X = L^{-1}: lane c solves L x = e_c (x_i = 0 for i < c), reading the
    // factor's rows back from shared memory.
    T x[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        T s = (i == lane) ? (T)1 : (T)0;
#pragma unroll
        for (int t = 0; t < i; ++t) s = fma(-B[i][t], x[t], s);
        const T ri = __shfl_sync(0xffffffffu, rdiag, i);
        x[i] = (i < kw && i >= lane) ? s * ri : (T)0;
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) Xs[i][lane] = (T)x[i];
    __syncwarp();
    return 0;
}

// The same factorisation and inverse spread over the whole CTA (used for
// FP64, whose per-warp issue rate is too low for one warp to carry it):
// right-looking column steps in shared memory, then X = L^{-1} by recursive
// doubling, X21 = -X22 (L21 X11), over blocks of size 1, 2, 4, 8, 16.
template <typename T>
__device__ int cta_chol_inv32(T (*B)[NB + 1], T (*Xs)[NB + 1], T (*Tt)[NB + 1], int kw,
                              double *ldiag) {
    __shared__ T rd[NB];
    __shared__ int fail_s;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) fail_s = 0;
    __syncthreads();
    for (int j = 0; j < kw; ++j) {
        if (tid == 0) {
            const T d = B[j][j];
            if (!(d > (T)0)) {
                fail_s = j + 1;
            } else {
                const T r = rsqrt_newton(d);
                B[j][j] = d * r;
                rd[j] = r;
                if (ldiag) ldiag[j] = (double)(d * r);
            }
        }
        __syncthreads();
        if (fail_s) return fail_s;
        const T r = rd[j];
        for (int i = j + 1 + tid; i < kw; i += nt) B[i][j] *= r;
        __syncthreads();
        const int rem = kw - j - 1;
        for (int idx = tid; idx < rem * rem; idx += nt) {
            const int i = j + 1 + idx / rem, c = j + 1 + idx % rem;
            if (c <= i) B[i][c] = fma(-B[i][j], B[c][j], B[i][c]);
        }
        __syncthreads();
    }
    for (int idx = tid; idx < NB * NB; idx += nt) {
        const int r = idx / NB, c = idx % NB;
        Xs[r][c] = (r == c && r < kw) ? rd[r] : (T)0;
        if (r >= kw || c > r) B[r][c] = (T)0;
    }
    __syncthreads();
    for (int h = 1; h < NB; h *= 2) {
        // pair p: rows/cols [2hp, 2hp + 2h); X11 = [2hp, 2hp+h), X22 = [2hp+h, 2hp+2h)
        const int per = h * h, total = (NB / (2 * h)) * per;
        for (int idx = tid; idx < total; idx += nt) {  // Tt = L21 X11
            const int p = idx / per, q = idx % per, k = q / h, c = q % h;
            const int r0 = 2 * h * p, row = r0 + h + k, col = r0 + c;
            T acc = 0;
            for (int m = col; m < r0 + h; ++m) acc = fma(B[row][m], Xs[m][col], acc);
            Tt[row][col] = acc;
        }
        __syncthreads();
        for (int idx = tid; idx < total; idx += nt) {  // X21 = -X22 Tt
            const int p = idx / per, q = idx % per, k = q / h, c = q % h;
            const int r0 = 2 * h * p, row = r0 + h + k, col = r0 + c;
            T acc = 0;
            for (int m = r0 + h; m <= row; ++m) acc = fma(Xs[row][m], Tt[m][col], acc);
            Xs[row][col] = -acc;
        }
        __syncthreads();
    }
    return 0;
}

template <typename T>
__device__ __forceinline__ int block_chol_inv32(T (*B)[NB + 1], T (*Xs)[NB + 1], T (*Tt)[NB + 1],
                                                int kw, double *ldiag) {
    if (sizeof(T) == 8) return cta_chol_inv32<T>(B, Xs, Tt, kw, ldiag);
    int f = 0;
    if (threadIdx.x < 32) f = warp_chol_inv32<T>(B, Xs, kw, ldiag);
    __shared__ int fshare;
    if (threadIdx.x == 0) fshare = f;
    __syncthreads();
    return fshare;
}

// Factor diagonal block kb (used for the first block) and store L_kk, X_kk.
template <typename T>
__global__ void __launch_bounds__(TPB) k_potrf_diag(T *__restrict__ A, int64_t n, int kb,
                                                    T *__restrict__ xd, double *__restrict__ ldiag,
                                                    DevScalars *sc) {
    if (sc->info != 0) return;
    __shared__ T B[NB][NB + 1], Xs[NB][NB + 1], Tt[NB][NB + 1];
    const int64_t k0 = (int64_t)kb * NB;
    const int kw = (int)lmin(NB, n - k0);
    for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
        const int r = idx / NB, c = idx % NB;
        B[r][c] = (r < kw && c <= r) ? A[(k0 + r) * n + k0 + c] : (T)0;
    }
    __syncthreads();
    const int f = block_chol_inv32<T>(B, Xs, Tt, kw, ldiag + k0);
    if (f) {
        if (threadIdx.x == 0) sc->info = (int)(k0 + f);
        return;
    }
    __syncthreads();
    T *X = xd + (kb & 1) * NB * NB;
    for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
        const int r = idx / NB, c = idx % NB;
        X[r * NB + c] = Xs[r][c];
        if (r < kw && c <= r) A[(k0 + r) * n + k0 + c] = B[r][c];
    }
}

// Panel of step kb: block row kb + 1 + blockIdx.x, L_ik = A_ik X_kk^T.
template <typename T>
__global__ void __launch_bounds__(TPB) k_potrf_panel(T *__restrict__ A, int64_t n, int kb,
                                                     const T *__restrict__ xd, DevScalars *sc) {
    if (sc->info != 0) return;
    __shared__ T As[NB][NB + 1], Bs[NB][NB + 1];
    const int64_t k0 = (int64_t)kb * NB;
    const int64_t kw = lmin(NB, n - k0);
    const int64_t i0 = k0 + (int64_t)(blockIdx.x + 1) * NB;
    const T *X = xd + (kb & 1) * NB * NB;
    T acc[2][2] = {{0, 0}, {0, 0}};
    // opA(i, c) = A[i0 + i, k0 + c]; opB(c, j) = X[j][c]
    tile_acc<T, false, true, T>(acc, A + i0 * n + k0, n, X, NB, 0, 0, 0, kw, n - i0, kw, As, Bs);
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int64_t i = i0 + ty + 16 * a, j = tx + 16 * b;
            if (i < n && j < kw) A[i * n + k0 + j] = acc[a][b];
        }
}

// Trailing update of step kb on lower tiles I >= J > kb; the CTA of tile
// (kb+1, kb+1) then factors that block and inverts its factor.
template <typename T>
__global__ void __launch_bounds__(TPB, 2) k_potrf_trail(T *__restrict__ A, int64_t n, int kb,
                                                     T *__restrict__ xd, double *__restrict__ ldiag,
                                                     DevScalars *sc) {
    if (sc->info != 0) return;
    __shared__ T As[NB][NB + 1], Bs[NB][NB + 1];
    int64_t I, J;
    tri_index(blockIdx.x, I, J);
    I += kb + 1;
    J += kb + 1;
    const int64_t k0 = (int64_t)kb * NB, k1 = lmin(k0 + NB, n);
    T acc[2][2] = {{0, 0}, {0, 0}};
    tile_acc<T, false, true, T>(acc, A, n, A, n, I * NB, J * NB, k0, k1, n, n, As, Bs);
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    const bool diag_next = (I == kb + 1 && J == kb + 1);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int64_t i = I * NB + ty + 16 * a, j = J * NB + tx + 16 * b;
            if (i < n && j < n && j <= i) {
                const T v = A[i * n + j] - acc[a][b];
                A[i * n + j] = v;
                if (diag_next) As[ty + 16 * a][tx + 16 * b] = v;
            }
        }
    if (!diag_next) return;
    __syncthreads();
    __shared__ T Tt[NB][NB + 1];
    const int64_t d0 = I * NB;
    const int kw = (int)lmin(NB, n - d0);
    const int f = block_chol_inv32<T>(As, Bs, Tt, kw, ldiag + d0);
    if (f) {
        if (threadIdx.x == 0) sc->info = (int)(d0 + f);
        return;
    }
    __syncthreads();
    T *X = xd + (I & 1) * NB * NB;
    for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
        const int r = idx / NB, c = idx % NB;
        X[r * NB + c] = Bs[r][c];
        if (r < kw && c <= r) A[(d0 + r) * n + d0 + c] = As[r][c];
    }
}

// Leaf of the tensor-core factorisation as a kernel of its own: one CTA of
// leaf::LT threads (see leaf32.cuh); a failing pivot goes to sc->info as its
// global index + 1, an expired wait to sc->tc_err.
__global__ void __launch_bounds__(leaf::LT, 1) k_leaf32(const float *__restrict__ A, int64_t ld, int64_t o,
                                                        int s, float *__restrict__ Xo,
                                                        float *__restrict__ Xto, double *__restrict__ ldiag,
                                                        DevScalars *sc) {
    pdl_wait();  // the block comes from the preceding kernel
    pdl_trigger();
    if (sc->info != 0) return;
    extern __shared__ float lsm[];
    __shared__ leaf::LeafShared lsh;
    const int f = leaf::leaf_factor(A, ld, o, s, Xo, ldiag, lsm, &lsh, 2000000000ll);
    if (f == 0) {
        leaf::leaf_store_xt(ld, o, s, Xto, lsm);
    } else if (threadIdx.x == 0) {
        if (f > 0) atomicCAS(&sc->info, 0, (int)(o + f));
        else atomicCAS(&sc->tc_err, 0, 19);
    }
}

// log det A = 2 sum_i log L_ii from the FP64 diagonal of the factor,
// deterministic single-CTA reduction.
__global__ void k_logdet(const double *__restrict__ ldiag, int64_t n, DevScalars *sc) {
    __shared__ double red[TPB];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += TPB) s += log(ldiag[i]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = TPB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) sc->logdet = (sc->info == 0) ? 2.0 * red[0] : 0.0;
}

// ---------------------------------------------------------------- a3: inverse
// Invert every 32 x 32 diagonal block of L: X_bb = L_bb^{-1} (forward
// substitution in FP64, one thread per column).
template <typename T>
__global__ void k_trtri_diag(const T *__restrict__ L, int64_t n, T *__restrict__ X) {
    __shared__ double Ls[NB][NB + 1];
    __shared__ double Xs[NB][NB + 1];
    const int64_t b0 = (int64_t)blockIdx.x * NB;
    const int bw = (int)lmin(NB, n - b0);
    for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
        int r = idx / NB, c = idx % NB;
        Ls[r][c] = (r < bw && c <= r) ? (double)L[(b0 + r) * n + b0 + c] : 0.0;
        Xs[r][c] = 0.0;
    }
    __syncthreads();
    const int c = threadIdx.x;
    if (c < bw) {
        for (int i = c; i < bw; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int t = c; t < i; ++t) s -= Ls[i][t] * Xs[t][c];
            Xs[i][c] = s / Ls[i][i];
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < bw * bw; idx += blockDim.x) {
        int r = idx / bw, cc = idx % bw;
        if (cc <= r) X[(b0 + r) * n + b0 + cc] = (T)Xs[r][cc];
    }
}

// Recursive doubling of the inverted diagonal blocks: for blocks of size s,
// pair p covers rows [r0, r0 + s + h) with r0 = 2 s p and
//   X21 = -X22 (L21 X11),  computed as  Tw = L21 X11, then X21 = -X22 Tw.
// Step 1: Tw_p (h x s, row stride s) = L21 X11; X11 is lower, so column
// block J only needs k >= J*32.
template <typename T>
__global__ void __launch_bounds__(TPB) k_trtri_step1(const T *__restrict__ L,
                                                     const T *__restrict__ X, int64_t n,
                                                     int64_t s, int tiles_i, int tiles_j,
                                                     T *__restrict__ Tw) {
    __shared__ T As[NB][NB + 1], Bs[NB][NB + 1];
    const int per = tiles_i * tiles_j;
    const int64_t p = blockIdx.x / per;
    const int tt = blockIdx.x % per;
    const int64_t I = tt / tiles_j, J = tt % tiles_j;
    const int64_t r0 = 2 * s * p;
    const int64_t h = lmin(s, n - r0 - s);
    if (I * NB >= h) return;
    T acc[2][2] = {{0, 0}, {0, 0}};
    tile_acc<T, false, false, T>(acc, L + (r0 + s) * n + r0, n, X + r0 * n + r0, n, I * NB,
                                 J * NB, J * NB, s, h, s, As, Bs);
    T *Tp = Tw + p * s * s;
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            int64_t i = I * NB + ty + 16 * a, j = J * NB + tx + 16 * b;
            if (i < h && j < s) Tp[i * s + j] = acc[a][b];
        }
}

// Step 2: X21 = -X22 Tw_p; X22 is lower, so row block I only needs k < (I+1)*32.
template <typename T>
__global__ void __launch_bounds__(TPB) k_trtri_step2(T *__restrict__ X, int64_t n, int64_t s,
                                                     int tiles_i, int tiles_j,
                                                     const T *__restrict__ Tw) {
    __shared__ T As[NB][NB + 1], Bs[NB][NB + 1];
    const int per = tiles_i * tiles_j;
    const int64_t p = blockIdx.x / per;
    const int tt = blockIdx.x % per;
    const int64_t I = tt / tiles_j, J = tt % tiles_j;
    const int64_t r0 = 2 * s * p;
    const int64_t h = lmin(s, n - r0 - s);
    if (I * NB >= h) return;
    const T *Tp = Tw + p * s * s;
    T acc[2][2] = {{0, 0}, {0, 0}};
    tile_acc<T, false, false, T>(acc, X + (r0 + s) * n + (r0 + s), n, Tp, s, I * NB, J * NB, 0,
                                 lmin((I + 1) * NB, h), h, s, As, Bs);
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            int64_t i = I * NB + ty + 16 * a, j = J * NB + tx + 16 * b;
            if (i < h && j < s) X[(r0 + s + i) * n + r0 + j] = -acc[a][b];
        }
}

// W = X^T X with X = L^{-1} lower: W_IJ = sum_{k >= I*32} X[k, I]^T X[k, J]
// on lower tiles I >= J, mirrored to the upper triangle.
template <typename T>
__global__ void __launch_bounds__(TPB) k_lauum(const T *__restrict__ X, int64_t n,
                                               T *__restrict__ W) {
    __shared__ T As[NB][NB + 1], Bs[NB][NB + 1];
    int64_t I, J;
    tri_index(blockIdx.x, I, J);
    T acc[2][2] = {{0, 0}, {0, 0}};
    tile_acc<T, true, false, T>(acc, X, n, X, n, I * NB, J * NB, I * NB, n, n, n, As, Bs);
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            int64_t i = I * NB + ty + 16 * a, j = J * NB + tx + 16 * b;
            if (i < n && j < n) {
                W[i * n + j] = acc[a][b];
                W[j * n + i] = acc[a][b];
            }
        }
}

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t form_S(const void *X, int dtype, int64_t m, int64_t n, int center, double *S,
                   double *Xstage, cudaStream_t st) {
    if (m < 1 || n < 1) return cudaErrorInvalidValue;
    // Xstage holds m*n + n doubles: the centred FP64 copy of X and the mean.
    // center == 2 computes the column means only (into Xstage + m*n).
    double *mu = center ? Xstage + m * n : nullptr;
    if (center == 2) {
        if (dtype == GLASSO_F64)
            k_colmean<double><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const double *)X, m, n, mu);
        else
            k_colmean<float><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const float *)X, m, n, mu);
        counted(1);
        return cudaGetLastError();
    }
    int g = (int)lmin((m * n + 255) / 256, 152 * 16);
    if (dtype == GLASSO_F64) {
        const double *x = (const double *)X;
        if (center) {
            k_colmean<double><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, m, n, mu);
            counted(1);
        }
        k_stage_x<double><<<g, 256, 0, st>>>(x, m, n, mu, Xstage);
        counted(1);
    } else {
        const float *x = (const float *)X;
        if (center) {
            k_colmean<float><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, m, n, mu);
            counted(1);
        }
        k_stage_x<float><<<g, 256, 0, st>>>(x, m, n, mu, Xstage);
        counted(1);
    }
    int64_t nb = (n + NB - 1) / NB;
    k_syrk_S<<<(unsigned)(nb * (nb + 1) / 2), TPB, 0, st>>>(Xstage, m, n, S);
    counted(1);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t potrf_t(T *A, int64_t n, T *xd, double *ldiag, DevScalars *sc, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(&sc->info, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const int64_t nb = (n + NB - 1) / NB;
    k_potrf_diag<T><<<1, TPB, 0, st>>>(A, n, 0, xd, ldiag, sc);
    counted(1);
    for (int64_t kb = 0; kb + 1 < nb; ++kb) {
        const int64_t m = nb - kb - 1;
        k_potrf_panel<T><<<(unsigned)m, TPB, 0, st>>>(A, n, (int)kb, xd, sc);
        k_potrf_trail<T><<<(unsigned)(m * (m + 1) / 2), TPB, 0, st>>>(A, n, (int)kb, xd, ldiag, sc);
        counted(2);
    }
    k_logdet<<<1, TPB, 0, st>>>(ldiag, n, sc);
    counted(1);
    return cudaGetLastError();
}

cudaError_t potrf(double *A, int64_t n, double *xd, double *ldiag, DevScalars *sc, cudaStream_t st) {
    return potrf_t<double>(A, n, xd, ldiag, sc, st);
}
cudaError_t potrf32(float *A, int64_t n, float *xd, double *ldiag, DevScalars *sc, cudaStream_t st) {
    return potrf_t<float>(A, n, xd, ldiag, sc, st);
}

template <typename T>
static cudaError_t inverse_t(const T *L, int64_t n, T *W, T *X, T *Tw, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(X, 0, (size_t)(n * n) * sizeof(T), st);
    if (e != cudaSuccess) return e;
    const int64_t nb = (n + NB - 1) / NB;
    k_trtri_diag<T><<<(unsigned)nb, NB, 0, st>>>(L, n, X);
    counted(1);
    for (int64_t s = NB; s < n; s *= 2) {
        const int64_t npairs = (n - s + 2 * s - 1) / (2 * s);  // r0 = 2sp with r0 + s < n
        const int tiles = (int)(s / NB);
        const unsigned grid = (unsigned)(npairs * tiles * tiles);
        k_trtri_step1<T><<<grid, TPB, 0, st>>>(L, X, n, s, tiles, tiles, Tw);
        k_trtri_step2<T><<<grid, TPB, 0, st>>>(X, n, s, tiles, tiles, Tw);
        counted(2);
    }
    k_lauum<T><<<(unsigned)(nb * (nb + 1) / 2), TPB, 0, st>>>(X, n, W);
    counted(1);
    return cudaGetLastError();
}

cudaError_t inverse(const double *L, int64_t n, double *W, double *X, double *Tw, cudaStream_t st) {
    return inverse_t<double>(L, n, W, X, Tw, st);
}
cudaError_t inverse32(const float *L, int64_t n, float *W, float *X, float *Tw, cudaStream_t st) {
    return inverse_t<float>(L, n, W, X, Tw, st);
}

cudaError_t chol_leaf32(const float *A, int64_t ld, int64_t o, int s, float *X, float *Xt, double *ldiag,
                        DevScalars *sc, cudaStream_t st) {
    static OncePerDevice once;
    int dev = 0;
    cudaError_t ie = once.run(dev, [](int) {
        return cudaFuncSetAttribute(k_leaf32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)leaf::LEAF_SMEM);
    });
    if (ie != cudaSuccess) return ie;
    if (s < 1 || s > leaf::LB) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};  // programmatic serialisation, as for the GEMMs
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(leaf::LT);
    cfg.dynamicSmemBytes = leaf::LEAF_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    la[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = la;
    cfg.numAttrs = 1;
    cudaError_t le = cudaLaunchKernelEx(&cfg, k_leaf32, A, ld, o, s, X, Xt, ldiag, sc);
    counted(1);
    path_hit(GLASSO_PATH_TC_LEAVES);
    if (le != cudaSuccess) return le;
    return cudaGetLastError();
}

cudaError_t logdet_from_diag(const double *ldiag, int64_t n, DevScalars *sc, cudaStream_t st) {
    k_logdet<<<1, TPB, 0, st>>>(ldiag, n, sc);
    counted(1);
    return cudaGetLastError();
}

}  // namespace glx
