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

__device__ __forceinline__ float rsqrt_newton(float d) {
    float r = rsqrtf(d);
    return r * fmaf(-0.5f * d * r, r, 1.5f);
}

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

// Leaf of the tensor-core factorisation (FP32): one CTA factors and inverts
// the diagonal block [o, o + s), s <= 128, of A (row stride ld) in shared
// memory.  L in 32-wide steps: each diagonal 32 x 32 block and its inverse by
// one warp in 8-wide sub-steps (warp_chol_inv32_blk; column-at-a-time forms,
// one warp or the whole CTA, took about 18 us per block on this GPU), then the
// panel L_ib = A_ib X_kk^T and the trailing update by the CTA; then X = L^{-1}
// by block substitution,
//   X_ij = -X_ii sum_{k=j}^{i-1} L_ik X_kj   (32-blocks, i > j),
// with the inner sums parked in the free upper blocks.  Rows beyond s are
// identity.  Writes the s x s blocks of X (lower, zeros above) and Xt = X^T
// (upper, zeros below), the FP64 diagonal of L into ldiag[o ..], and the first
// failing pivot + 1 (global index) into sc->info.  The CTA-wide products keep
// several independent accumulators per thread (register tiles): this kernel
// runs once per leaf on one SM, so its latency is what counts.
constexpr int LB = 128, LP = LB + 1;
constexpr size_t LEAF_SMEM = 2 * LB * LP * sizeof(float);

// One thread: Cholesky of the 8 x 8 lower block a (registers) in place and
// x = L^{-1}; rd[i] = 1 / L_ii.  Returns 0 or the failing pivot + 1.
__device__ __forceinline__ int thread_chol_inv8(float (&a)[8][8], float (&x)[8][8], float (&rd)[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float d = a[j][j];
        if (!(d > 0.f)) return j + 1;
        const float r = rsqrt_newton(d);
        rd[j] = r;
        a[j][j] = d * r;
#pragma unroll
        for (int i = j + 1; i < 8; ++i) a[i][j] *= r;
#pragma unroll
        for (int i = j + 1; i < 8; ++i)
#pragma unroll
            for (int k = j + 1; k <= i; ++k) a[i][k] = fmaf(-a[i][j], a[k][j], a[i][k]);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i < c) {
                x[i][c] = 0.f;
            } else {
                float s = (i == c) ? 1.f : 0.f;
#pragma unroll
                for (int t = c; t < i; ++t) s = fmaf(-a[i][t], x[t][c], s);
                x[i][c] = s * rd[i];
            }
        }
    return 0;
}

// One warp: Cholesky of the 32 x 32 block B (lower, row stride NB + 1) in
// place and Xs = L^{-1}, both with zero upper triangles, in 8-wide steps: one
// lane factors and inverts each 8 x 8 diagonal block in registers, the warp
// forms the sub-panel (L_ik = A_ik X_kk^T) and the trailing update; then the
// off-diagonal 8-blocks of the inverse by substitution,
// X_ij = -X_ii sum_{k=j}^{i-1} L_ik X_kj.  The serial path is four 8 x 8
// factorisations, not 32 dependent column steps.  Returns 0 or pivot + 1.
__device__ int warp_chol_inv32_blk(float (*B)[NB + 1], float (*Xs)[NB + 1], int *fflag) {
    const int lane = threadIdx.x & 31;
    for (int kb = 0; kb < 4; ++kb) {
        const int o = 8 * kb;
        if (lane == 0) {
            float a[8][8], x[8][8], rd[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) a[i][j] = (j <= i) ? B[o + i][o + j] : 0.f;
            const int f = thread_chol_inv8(a, x, rd);
            *fflag = f ? o + f : 0;
            if (!f) {
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        B[o + i][o + j] = (j <= i) ? a[i][j] : 0.f;
                        Xs[o + i][o + j] = x[i][j];
                    }
            }
        }
        __syncwarp();
        const int f = *fflag;
        if (f) return f;
        const int rows = NB - o - 8;  // rows below the diagonal block
        if (rows == 0) break;
        // sub-panel: L[r][o + c] = sum_{t <= c} B[r][o + t] Xs[o + c][o + t]
        float pv[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int idx = lane + 32 * q;
            pv[q] = 0.f;
            if (idx < rows * 8) {
                const int r = o + 8 + idx / 8, c = idx % 8;
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (t <= c) acc = fmaf(B[r][o + t], Xs[o + c][o + t], acc);
                pv[q] = acc;
            }
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int idx = lane + 32 * q;
            if (idx < rows * 8) B[o + 8 + idx / 8][o + idx % 8] = pv[q];
        }
        __syncwarp();
        // trailing update: lane owns column j = o + 8 + lane, rows i >= j
        if (lane < rows) {
            const int j = o + 8 + lane;
            float lj[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) lj[t] = B[j][o + t];
            for (int i = j; i < NB; ++i) {
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t < 8; ++t) acc = fmaf(B[i][o + t], lj[t], acc);
                B[i][j] -= acc;
            }
        }
        __syncwarp();
    }
    // off-diagonal 8-blocks of the inverse, by block distance
    for (int diff = 1; diff < 4; ++diff) {
        const int nblk = 4 - diff;
        // T_ij = sum_{k = 8 jb}^{8 ib - 1} L[8 ib + r][k] X[k][8 jb + c], parked in the upper block
        float tv[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int idx = lane + 32 * q;
            tv[q] = 0.f;
            if (idx < nblk * 64) {
                const int jb = idx / 64, r = (idx / 8) % 8, c = idx % 8, ib = jb + diff;
                float acc = 0.f;
                for (int k = 8 * jb; k < 8 * ib; ++k) acc = fmaf(B[8 * ib + r][k], Xs[k][8 * jb + c], acc);
                tv[q] = acc;
            }
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int idx = lane + 32 * q;
            if (idx < nblk * 64) {
                const int jb = idx / 64, r = (idx / 8) % 8, c = idx % 8, ib = jb + diff;
                Xs[8 * jb + r][8 * ib + c] = tv[q];
            }
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int idx = lane + 32 * q;
            if (idx < nblk * 64) {
                const int jb = idx / 64, r = (idx / 8) % 8, c = idx % 8, ib = jb + diff;
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (t <= r) acc = fmaf(Xs[8 * ib + r][8 * ib + t], Xs[8 * jb + t][8 * ib + c], acc);
                tv[q] = -acc;
            }
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int idx = lane + 32 * q;
            if (idx < nblk * 64) {
                const int jb = idx / 64, r = (idx / 8) % 8, c = idx % 8, ib = jb + diff;
                Xs[8 * ib + r][8 * jb + c] = tv[q];
            }
        }
        __syncwarp();
    }
    // zero the upper triangle of the inverse (it held the parked sums)
    for (int idx = lane; idx < NB * NB; idx += 32) {
        const int r = idx / NB, c = idx % NB;
        if (c > r) Xs[r][c] = 0.f;
    }
    __syncwarp();
    return 0;
}

// Trailing update of the m x m block below and right of step d0 (m = 96, 64,
// 32): L[i][j] -= sum_t L[i][d0+t] L[j][d0+t], lower part; thread (warp w,
// lane c) owns rows w + 8 q and columns c + 32 p.
template <int M>
__device__ __forceinline__ void leaf_trail(float (*L)[LP], int d0) {
    constexpr int NQ = M / 8, NPC = M / 32;
    const int w = threadIdx.x >> 5, c = threadIdx.x & 31, b0 = d0 + NB;
    float acc[NQ][NPC];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int p = 0; p < NPC; ++p) acc[q][p] = 0.f;
#pragma unroll 4
    for (int t = 0; t < NB; ++t) {
        float lj[NPC], li[NQ];
#pragma unroll
        for (int p = 0; p < NPC; ++p) lj[p] = L[b0 + c + 32 * p][d0 + t];
#pragma unroll
        for (int q = 0; q < NQ; ++q) li[q] = L[b0 + w + 8 * q][d0 + t];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int p = 0; p < NPC; ++p) acc[q][p] = fmaf(li[q], lj[p], acc[q][p]);
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int p = 0; p < NPC; ++p) {
            const int i = b0 + w + 8 * q, j = b0 + c + 32 * p;
            if (j <= i) L[i][j] -= acc[q][p];
        }
}

__global__ void __launch_bounds__(TPB, 1) k_leaf32(const float *__restrict__ A, int64_t ld, int64_t o,
                                                    int s, float *__restrict__ Xo,
                                                    float *__restrict__ Xto, double *__restrict__ ldiag,
                                                    DevScalars *sc) {
    if (sc->info != 0) return;
    extern __shared__ float lsm[];
    float(*L)[LP] = reinterpret_cast<float(*)[LP]>(lsm);
    float(*X)[LP] = reinterpret_cast<float(*)[LP]>(lsm + LB * LP);
    __shared__ float B[NB][NB + 1], Xd[NB][NB + 1];
    __shared__ int fshare, fflag;
    const int tid = threadIdx.x, w = tid >> 5, c = tid & 31;
    for (int idx = tid; idx < LB * LB; idx += TPB) {
        const int r = idx / LB, cc = idx % LB;
        float v = 0.f;
        if (r < s && cc <= r) v = A[(o + r) * ld + o + cc];
        else if (r == cc) v = 1.f;
        L[r][cc] = v;
        X[r][cc] = 0.f;
    }
    __syncthreads();
    for (int kb = 0; kb < LB / NB; ++kb) {
        const int d0 = kb * NB;
        for (int idx = tid; idx < NB * NB; idx += TPB) B[idx / NB][idx % NB] = L[d0 + idx / NB][d0 + idx % NB];
        __syncthreads();
        if (w == 0) {
            const int f = warp_chol_inv32_blk(B, Xd, &fflag);
            if (c == 0) fshare = f;
        }
        __syncthreads();
        if (fshare) {
            if (tid == 0) atomicCAS(&sc->info, 0, (int)(o + d0 + fshare));
            return;
        }
        for (int idx = tid; idx < NB * NB; idx += TPB) {
            const int r = idx / NB, cc = idx % NB;
            L[d0 + r][d0 + cc] = B[r][cc];
            X[d0 + r][d0 + cc] = Xd[r][cc];
        }
        const int nrem = LB / NB - kb - 1;
        if (nrem == 0) break;
        // panel: L[row][d0 + c] = sum_{t <= c} L[row][d0 + t] Xd[c][t]; thread
        // (warp w, lane c) owns rows d0 + 32 + w + 8 q
        {
            float acc[12];
#pragma unroll
            for (int q = 0; q < 12; ++q) acc[q] = 0.f;
            const int rows = nrem * NB;
            for (int t = 0; t <= c; ++t) {
                const float xc = Xd[c][t];
#pragma unroll
                for (int q = 0; q < 12; ++q)
                    if (w + 8 * q < rows) acc[q] = fmaf(L[d0 + NB + w + 8 * q][d0 + t], xc, acc[q]);
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 12; ++q)
                if (w + 8 * q < rows) L[d0 + NB + w + 8 * q][d0 + c] = acc[q];
        }
        __syncthreads();
        if (kb == 0) leaf_trail<96>(L, d0);
        else if (kb == 1) leaf_trail<64>(L, d0);
        else leaf_trail<32>(L, d0);
        __syncthreads();
    }
    for (int r = tid; r < s; r += TPB) ldiag[o + r] = (double)L[r][r];
    // X below the diagonal blocks, by distance of block row and column; thread
    // (warp w, lane c) owns rows w + 8 q (q < 4) of each block in the step
    for (int diff = 1; diff < LB / NB; ++diff) {
        const int nblk = LB / NB - diff;
        for (int jb = 0; jb < nblk; ++jb) {
            const int ib = jb + diff;
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k = jb * NB; k < ib * NB; ++k) {
                const float xk = X[k][jb * NB + c];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = fmaf(L[ib * NB + w + 8 * q][k], xk, acc[q]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) X[jb * NB + w + 8 * q][ib * NB + c] = acc[q];  // T_ij, parked
        }
        __syncthreads();
        for (int jb = 0; jb < nblk; ++jb) {
            const int ib = jb + diff;
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int t = 0; t < NB; ++t) {
                const float tv = X[jb * NB + t][ib * NB + c];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int r = w + 8 * q;
                    if (t <= r) acc[q] = fmaf(X[ib * NB + r][ib * NB + t], tv, acc[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) X[ib * NB + w + 8 * q][jb * NB + c] = -acc[q];
        }
        __syncthreads();
    }
    for (int idx = tid; idx < s * s; idx += TPB) {
        const int r = idx / s, cc = idx % s;
        Xo[(o + r) * ld + o + cc] = (cc <= r) ? X[r][cc] : 0.f;
        Xto[(o + r) * ld + o + cc] = (cc >= r) ? X[cc][r] : 0.f;
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
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_leaf32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)LEAF_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (s < 1 || s > LB) return cudaErrorInvalidValue;
    k_leaf32<<<1, TPB, LEAF_SMEM, st>>>(A, ld, o, s, X, Xt, ldiag, sc);
    counted(1);
    return cudaGetLastError();
}

cudaError_t logdet_from_diag(const double *ldiag, int64_t n, DevScalars *sc, cudaStream_t st) {
    k_logdet<<<1, TPB, 0, st>>>(ldiag, n, sc);
    counted(1);
    return cudaGetLastError();
}

}  // namespace glx
