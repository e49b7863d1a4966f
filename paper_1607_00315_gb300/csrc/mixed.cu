// Kernels of the mixed-precision relaxation.
//
// The bulk arithmetic moves to FP32 / TF32 while the quantities that decide
// the answer stay FP64:
//  * W = A^{-1} is refined against A by Newton-Schulz steps
//        R = I - A W            (A sparse: CSR of its nonzeros)
//        W <- W + W R           (TF32 tensor-core GEMM of the small correction,
//                                tc.cu)
//    until |R| reaches 1e-11, and then rounded to FP64; the gradient S - W,
//    the free set and the KKT residual therefore see an FP64-accurate W (eq.
//    gradHes, eq. active_set, the Section 8 stopping rule).  During the
//    refinement W is a pair of FP32 arrays, W = hi + lo (|lo| <= ulp(hi) / 2,
//    about 48 significant bits), and R and the update are formed with
//    error-free products and sums in FP32 (FP64 arithmetic runs at a small
//    fraction of the FP32 rate on this GPU): per term, a_hi w_hi = p + e
//    exactly (p rounded, e = fma(a_hi, w_hi, -p)), the cross terms a_hi w_lo +
//    a_lo w_hi in FP32 (relative 2^-48 of the product), and the running sum
//    kept as hi + lo with Knuth's two-sum.
//  * The line search (Section 6.1.2) gets log det(A + alpha Delta) - log det A
//    from the series  sum_k (-1)^{k+1} alpha^k t_k / k,  t_k = tr((W Delta)^k):
//    t1 on the pairs (FP64), t2 = sum U_kj U_jk with U = Delta W from the
//    sweep, t3 .. t6 from U^2 and U^3 on the tensor cores; the remainder after
//    K terms is at most rho^{K+1} / ((K+1)(1 - rho)), rho = alpha sqrt(t2), and
//    rho < 1 also proves A + alpha Delta positive definite.  Large steps use an
//    FP32 Cholesky (FP64 log accumulation) instead.
#include <math.h>

#include "glasso_internal.h"

namespace glx {
namespace {

__device__ __forceinline__ void tri_index64(int64_t t, int64_t &I, int64_t &J) {
    int64_t i = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > t) --i;
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    I = i;
    J = t - i * (i + 1) / 2;
}

// ---- CSR of the nonzeros of A (full rows, column order) --------------------
constexpr int RW = 8;  // rows (warps) per CTA

__global__ void k_nz_count(const double *__restrict__ A, int64_t n, long long *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * RW + (threadIdx.x >> 5);
    if (i >= n) return;
    long long c = 0;
    for (int64_t j0 = 0; j0 < n; j0 += 32) {
        const int64_t j = j0 + lane;
        const bool nz = j < n && A[i * n + j] != 0.0;
        c += __popc(__ballot_sync(0xffffffffu, nz));
    }
    if (lane == 0) cnt[i] = c;
}

__global__ void k_rowptr_scan(long long *__restrict__ cnt, int64_t n) {
    // one CTA of 1024 threads: exclusive scan in place, total at cnt[n]
    __shared__ long long part[1024];
    const int t = threadIdx.x;
    const int64_t per = (n + 1023) / 1024;
    const int64_t a = t * per, b = lmin(a + per, n);
    long long s = 0;
    for (int64_t i = a; i < b; ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        long long v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long off = part[t] - s;
    for (int64_t i = a; i < b; ++i) {
        const long long c = cnt[i];
        cnt[i] = off;
        off += c;
    }
    if (t == 1023) cnt[n] = part[1023];
}

__global__ void k_nz_write(const double *__restrict__ A, int64_t n, const long long *__restrict__ ptr,
                           int32_t *__restrict__ col, double *__restrict__ val) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * RW + (threadIdx.x >> 5);
    if (i >= n) return;
    long long off = ptr[i];
    for (int64_t j0 = 0; j0 < n; j0 += 32) {
        const int64_t j = j0 + lane;
        const double a = j < n ? A[i * n + j] : 0.0;
        const uint32_t m = __ballot_sync(0xffffffffu, a != 0.0);
        if (a != 0.0) {
            const long long pos = off + __popc(m & ((1u << lane) - 1u));
            col[pos] = (int32_t)j;
            val[pos] = a;
        }
        off += __popc(m);
    }
}

// ---- residual R = I - A W with W = hi + lo (double-float), per-row max and
// sum of squares of R (FP32; they decide convergence against 1e-11 and the
// restart at |R|_F >= 0.9).  The CSR values of A are split into FP32 pairs
// as they are staged.
constexpr int RES_T = 256;
constexpr int64_t SERIES_CTAS = 152 * 4;  // persistent CTAs of the series reductions
constexpr int RES_CAP = 256;  // nonzeros of a row staged per pass

__global__ void __launch_bounds__(RES_T) k_residual(const long long *__restrict__ ptr,
                                                    const int32_t *__restrict__ col,
                                                    const double *__restrict__ val,
                                                    const float *__restrict__ Whi,
                                                    const float *__restrict__ Wlo, int64_t n,
                                                    float *__restrict__ R32,
                                                    double *__restrict__ rowstat, DevScalars *dsc) {
    __shared__ int32_t sc[RES_CAP];
    __shared__ int last_s;
    __shared__ float sh[RES_CAP], sl[RES_CAP];
    __shared__ float rmax[RES_T], rsq[RES_T];
    const int64_t i = blockIdx.x;
    const long long p0 = ptr[i], p1 = ptr[i + 1];
    float mx = 0.f, sq = 0.f;
    // columns handled by this thread, in registers for up to 8 chunks of RES_T
    for (int64_t c0 = 0; c0 < n; c0 += (int64_t)RES_T * 8) {
        float ah[8], al[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t cidx = c0 + threadIdx.x + (int64_t)q * RES_T;
            ah[q] = (cidx == i) ? 1.f : 0.f;
            al[q] = 0.f;
        }
        for (long long pb = p0; pb < p1; pb += RES_CAP) {
            const int cntk = (int)lmin(RES_CAP, p1 - pb);
            __syncthreads();
            for (int t = threadIdx.x; t < cntk; t += RES_T) {
                const double a = val[pb + t];
                const float h = (float)a;
                sc[t] = col[pb + t];
                sh[t] = h;
                sl[t] = (float)(a - (double)h);
            }
            __syncthreads();
            // two nonzeros per step, all their W loads issued before the sums
            for (int t0 = 0; t0 < cntk; t0 += 2) {
                float x1[2][8], x2[2][8], a1[2], a2[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int t = t0 + u < cntk ? t0 + u : t0;  // (a repeated term gets a = 0)
                    a1[u] = t0 + u < cntk ? sh[t] : 0.f;
                    a2[u] = t0 + u < cntk ? sl[t] : 0.f;
                    const float *wh = Whi + (int64_t)sc[t] * n, *wl = Wlo + (int64_t)sc[t] * n;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int64_t cidx = c0 + threadIdx.x + (int64_t)q * RES_T;
                        x1[u][q] = cidx < n ? wh[cidx] : 0.f;
                        x2[u][q] = cidx < n ? wl[cidx] : 0.f;
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float pr = __fmul_rn(a1[u], x1[u][q]);
                        const float pe = fmaf(a1[u], x1[u][q], -pr);                     // a1 x1 = pr + pe
                        const float px = fmaf(a1[u], x2[u][q], __fmul_rn(a2[u], x1[u][q]));  // cross terms
                        // (ah, al) -= pr + (pe + px): two-sum of ah and -pr
                        const float sm = __fsub_rn(ah[q], pr);
                        const float bb = __fsub_rn(sm, ah[q]);
                        const float er = __fadd_rn(__fsub_rn(ah[q], __fsub_rn(sm, bb)), __fsub_rn(-pr, bb));
                        al[q] = __fadd_rn(al[q], __fsub_rn(er, __fadd_rn(pe, px)));
                        ah[q] = sm;
                    }
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t cidx = c0 + threadIdx.x + (int64_t)q * RES_T;
            if (cidx < n) {
                const float r = __fadd_rn(ah[q], al[q]);
                R32[i * n + cidx] = r;
                mx = fmaxf(mx, fabsf(r));
                sq = fmaf(r, r, sq);
            }
        }
    }
    rmax[threadIdx.x] = mx;
    rsq[threadIdx.x] = sq;
    __syncthreads();
    for (int w = RES_T / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            rmax[threadIdx.x] = fmaxf(rmax[threadIdx.x], rmax[threadIdx.x + w]);
            rsq[threadIdx.x] += rsq[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        rowstat[2 * i] = (double)rmax[0];
        rowstat[2 * i + 1] = (double)rsq[0];
        __threadfence();
        last_s = atomicAdd(&dsc->res_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last_s) return;
    // the last CTA: fixed-order reduction of the per-row (max, sum) pairs
    // into ns_max, ns_fro2 (L2 loads: the pairs were written by other SMs)
    __shared__ double m2[RES_T], s2[RES_T];
    double mxd = 0.0, sqd = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += RES_T) {
        mxd = fmax(mxd, __ldcg(rowstat + 2 * r));
        sqd += __ldcg(rowstat + 2 * r + 1);
    }
    m2[threadIdx.x] = mxd;
    s2[threadIdx.x] = sqd;
    __syncthreads();
    for (int w = RES_T / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            m2[threadIdx.x] = fmax(m2[threadIdx.x], m2[threadIdx.x + w]);
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        dsc->ns_max = m2[0];
        dsc->ns_fro2 = s2[0];
        dsc->res_done = 0u;  // ready for the next launch
    }
}

// W (FP64) -> hi = fl32(W), lo = fl32(W - hi); and back, W = hi + lo.
__global__ void k_split64(const double *__restrict__ W, float *__restrict__ hi, float *__restrict__ lo,
                          int64_t m) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double w = W[t];
        const float h = (float)w;
        hi[t] = h;
        lo[t] = (float)(w - (double)h);
    }
}

__global__ void k_join64(const float *__restrict__ hi, const float *__restrict__ lo, double *__restrict__ W,
                         int64_t m) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x)
        W[t] = (double)hi[t] + (double)lo[t];
}

// ---- t2 = tr((Delta W)^2) = sum_kj U_kj U_jk over 32 x 32 tile pairs -------
// Persistent CTAs walk the upper tile pairs (I <= J; the off-diagonal pairs
// count twice).  Each product is split exactly (p + e, e = fma(a, b, -p)) and
// summed in double-float FP32 (two-sum), so no FP64 arithmetic runs per
// element; each CTA's sum goes to part[] in FP64.
__device__ __forceinline__ void df_acc(float &h, float &l, float a, float b, float w) {
    const float p = __fmul_rn(a, b) * w, pe = fmaf(a, b, -__fmul_rn(a, b)) * w;  // w = 1 or 2 (exact)
    const float sm = __fadd_rn(h, p), bb = __fsub_rn(sm, h);
    const float er = __fadd_rn(__fsub_rn(h, __fsub_rn(sm, bb)), __fsub_rn(p, bb));
    l = __fadd_rn(l, __fadd_rn(er, pe));
    h = sm;
}

// block sum of (h + l) in FP64 (one value per thread), written by thread 0
__device__ __forceinline__ void df_block_sum(float h, float l, double *out) {
    __shared__ double wsum[8];
    double v = (double)h + (double)l;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
        *out = t;
    }
}

__global__ void k_t2_tiles(const float *__restrict__ U, int64_t n, double *__restrict__ part) {
    __shared__ float Ut[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 x 32
    const int64_t nt = (n + 31) / 32, ntiles = nt * (nt + 1) / 2;
    float h = 0.f, l = 0.f;
    for (int64_t q = blockIdx.x; q < ntiles; q += gridDim.x) {
        int64_t I, J;
        tri_index64(q, I, J);
        // stage U[J-block rows, I-block cols] transposed
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {
            const int64_t gr = J * 32 + r, gc = I * 32 + tx;
            Ut[tx][r] = (gr < n && gc < n) ? U[gr * n + gc] : 0.f;
        }
        __syncthreads();
        const float w = I == J ? 1.f : 2.f;
        for (int r = ty; r < 32; r += 8) {
            const int64_t gr = I * 32 + r, gc = J * 32 + tx;
            if (gr < n && gc < n) df_acc(h, l, U[gr * n + gc], Ut[r][tx], w);
        }
    }
    df_block_sum(h, l, part + blockIdx.x);
}

__global__ void k_sum_final(const double *__restrict__ part, int64_t m, double *out) {
    __shared__ double s[1024];
    const int t = threadIdx.x;
    double a = 0.0;
    for (int64_t i = t; i < m; i += 1024) a += part[i];
    s[t] = a;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (t < w) s[t] += s[t + w];
        __syncthreads();
    }
    if (t == 0) *out = s[0];
}

// sum_{i,j < n} P_ij Q_ji over all 32 x 32 tile pairs, persistent CTAs,
// products and sums as in k_t2_tiles; one FP64 partial per CTA
__global__ void k_tdot_tiles(const float *__restrict__ P, int64_t ldp_, const float *__restrict__ Q,
                             int64_t ldq, int64_t n, double *__restrict__ part) {
    __shared__ float Qt[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t nt = (n + 31) / 32;
    float h = 0.f, l = 0.f;
    for (int64_t q = blockIdx.x; q < nt * nt; q += gridDim.x) {
        const int64_t I = q / nt, J = q - (q / nt) * nt;
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {  // Qt[c][r] = Q[J*32 + r][I*32 + c]
            const int64_t gr = J * 32 + r, gc = I * 32 + tx;
            Qt[tx][r] = (gr < n && gc < n) ? Q[gr * ldq + gc] : 0.f;
        }
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {
            const int64_t gr = I * 32 + r, gc = J * 32 + tx;
            if (gr < n && gc < n) df_acc(h, l, P[gr * ldp_ + gc], Qt[r][tx], 1.f);
        }
    }
    df_block_sum(h, l, part + blockIdx.x);
}

// t1 = tr(W Delta) = sum over pairs of mult W_ij Delta_ij (FP64); per-block partials
__global__ void k_t1_part(const double *__restrict__ W64, int64_t n, const int32_t *__restrict__ pi,
                          const int32_t *__restrict__ pj, const double *__restrict__ D, int64_t np,
                          double *__restrict__ part) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t p = blockIdx.x * 256ll + threadIdx.x; p < np; p += (int64_t)gridDim.x * 256) {
        const int64_t i = pi[p], j = pj[p];
        s += (i == j ? 1.0 : 2.0) * W64[i * n + j] * D[p];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// ---- conversions and trial matrices -----------------------------------------
__global__ void k_to_f32(const double *__restrict__ x, float *__restrict__ y, int64_t m) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x)
        y[t] = (float)x[t];
}

__global__ void k_to_f64(const float *__restrict__ x, double *__restrict__ y, int64_t m) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x)
        y[t] = (double)x[t];
}

__global__ void k_scatter_f32(float *__restrict__ T, int64_t ldT, const int32_t *__restrict__ pi,
                              const int32_t *__restrict__ pj, const double *__restrict__ aval,
                              const double *__restrict__ D, int64_t np, double alpha) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = pi[p], j = pj[p];
        const float v = (float)(aval[p] + alpha * D[p]);
        T[i * ldT + j] = v;
        T[j * ldT + i] = v;
    }
}

// T[i][j] = (float)A[i][j] with row stride ldT.
__global__ void k_to_f32_ld(const double *__restrict__ A, int64_t n, float *__restrict__ T, int64_t ldT) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / n, j = t - i * n;
        T[i * ldT + j] = (float)A[t];
    }
}

// W64 = diag(1 / A_ii) for a diagonal A (the initial iterate), per-row log A_ii
__global__ void k_diag_inverse(const double *__restrict__ A, int64_t n, double *__restrict__ W64,
                               double *__restrict__ logs) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double a = A[i * n + i];
        W64[i * n + i] = 1.0 / a;
        logs[i] = log(a);
    }
}

inline unsigned gridn(int64_t work, int per = 256) {
    int64_t g = (work + per - 1) / per;
    return (unsigned)lmax(1, lmin(g, 152 * 16));
}

}  // namespace

cudaError_t build_csr(const double *A, int64_t n, long long *ptr, int32_t *col, double *val,
                      cudaStream_t st) {
    const unsigned g = (unsigned)((n + RW - 1) / RW);
    k_nz_count<<<g, 32 * RW, 0, st>>>(A, n, ptr);
    k_rowptr_scan<<<1, 1024, 0, st>>>(ptr, n);
    k_nz_write<<<g, 32 * RW, 0, st>>>(A, n, ptr, col, val);
    counted(3);
    return cudaGetLastError();
}

cudaError_t residual(const long long *ptr, const int32_t *col, const double *val, const float *Whi,
                     const float *Wlo, int64_t n, float *R32, double *rowstat, DevScalars *sc,
                     cudaStream_t st) {
    k_residual<<<(unsigned)n, RES_T, 0, st>>>(ptr, col, val, Whi, Wlo, n, R32, rowstat, sc);
    counted(1);
    return cudaGetLastError();
}

cudaError_t series_terms(const double *W64, int64_t n, const int32_t *pi, const int32_t *pj,
                         const double *D, int64_t np, const float *U32, double *part, int64_t cap,
                         DevScalars *sc, cudaStream_t st) {
    const int64_t nt = (n + 31) / 32;
    const int64_t ntiles = lmin(nt * (nt + 1) / 2, SERIES_CTAS);  // persistent CTAs
    const int nb1 = (int)lmin(1024, lmax(1, (np + 255) / 256));
    if (ntiles + nb1 > cap) return cudaErrorInvalidValue;
    k_t2_tiles<<<(unsigned)ntiles, 256, 0, st>>>(U32, n, part);
    k_sum_final<<<1, 1024, 0, st>>>(part, ntiles, &sc->t2);
    k_t1_part<<<nb1, 256, 0, st>>>(W64, n, pi, pj, D, np, part + ntiles);
    k_sum_final<<<1, 1024, 0, st>>>(part + ntiles, nb1, &sc->t1);
    counted(4);
    return cudaGetLastError();
}

// t3 .. t6 of the log-det series from U = Delta W (FP32, ld n):
//   t3 = sum (U^2)_ij U_ji, t4 = sum (U^2)_ij (U^2)_ji, t5 = sum (U^2)_ij (U^3)_ji,
//   t6 = sum (U^3)_ij (U^3)_ji, with U^2 and U^3 from TF32 tensor-core GEMMs.
// Up, Ut, U2, U3: scratch of tc_pad(n)^2 floats each.
cudaError_t series_high(const float *U32, int64_t n, float *Up, float *Ut, float *U2, float *U3,
                        double *part, int64_t cap, DevScalars *sc, cudaStream_t st) {
    const int64_t p = tc_pad(n);
    const int64_t nt = (n + 31) / 32;
    const int64_t nct = lmin(nt * nt, SERIES_CTAS);  // persistent CTAs
    if (nct > cap) return cudaErrorInvalidValue;
    cudaError_t e = pad_and_transpose(U32, n, Up, Ut, st);
    if (e != cudaSuccess) return e;
    // split-TF32 products with unbiased summation: the terms carry about
    // (n / 8 + 2) 2^-24 relative error, so the series is usable up to a
    // larger step than with single-TF32 products
    e = gemm_nt_split(Up, Ut, n, p, U2, &sc->tc_err, st);  // U^2
    if (e != cudaSuccess) return e;
    e = gemm_nt_split(U2, Ut, n, p, U3, &sc->tc_err, st);  // U^3
    if (e != cudaSuccess) return e;
    const float *Ps[4] = {U2, U2, U2, U3};
    const float *Qs[4] = {Up, U2, U3, U3};
    double *outs[4] = {&sc->t3, &sc->t4, &sc->t5, &sc->t6};
    for (int k = 0; k < 4; ++k) {
        k_tdot_tiles<<<(unsigned)nct, 256, 0, st>>>(Ps[k], p, Qs[k], p, n, part);
        k_sum_final<<<1, 1024, 0, st>>>(part, nct, outs[k]);
        counted(2);
    }
    return cudaGetLastError();
}

cudaError_t split64(const double *W, float *hi, float *lo, int64_t m, cudaStream_t st) {
    k_split64<<<gridn(m), 256, 0, st>>>(W, hi, lo, m);
    counted(1);
    return cudaGetLastError();
}

cudaError_t join64(const float *hi, const float *lo, double *W, int64_t m, cudaStream_t st) {
    k_join64<<<gridn(m), 256, 0, st>>>(hi, lo, W, m);
    counted(1);
    return cudaGetLastError();
}

cudaError_t to_f32(const double *x, float *y, int64_t m, cudaStream_t st) {
    k_to_f32<<<gridn(m), 256, 0, st>>>(x, y, m);
    counted(1);
    return cudaGetLastError();
}

cudaError_t to_f64(const float *x, double *y, int64_t m, cudaStream_t st) {
    k_to_f64<<<gridn(m), 256, 0, st>>>(x, y, m);
    counted(1);
    return cudaGetLastError();
}

cudaError_t trial32(const double *A, float *T, int64_t n, int64_t ldT, const int32_t *pi,
                    const int32_t *pj, const double *aval, const double *D, int64_t np, double alpha,
                    cudaStream_t st) {
    k_to_f32_ld<<<gridn(n * n), 256, 0, st>>>(A, n, T, ldT);
    counted(1);
    if (np > 0) {
        k_scatter_f32<<<gridn(np), 256, 0, st>>>(T, ldT, pi, pj, aval, D, np, alpha);
        counted(1);
    }
    return cudaGetLastError();
}

cudaError_t diag_inverse(const double *A, int64_t n, double *W64, double *logs, DevScalars *sc,
                         cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(W64, 0, (size_t)(n * n) * sizeof(double), st);
    if (e != cudaSuccess) return e;
    k_diag_inverse<<<gridn(n), 256, 0, st>>>(A, n, W64, logs);
    k_sum_final<<<1, 1024, 0, st>>>(logs, n, &sc->logdet);
    counted(2);
    return cudaGetLastError();
}

}  // namespace glx
