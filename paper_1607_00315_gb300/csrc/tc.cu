// TF32 tensor-core GEMM on the 5th-generation tensor cores (tcgen05):
//   C[i][j] = sum_k P[i][k] Q[j][k]      (both operands K-major, FP32 in HBM)
// on 128 x 128 output tiles, fed by TMA into 128-byte-swizzled shared-memory
// tiles through a 4-stage mbarrier pipeline, accumulated in TMEM by
// tcgen05.mma.kind::tf32 (M = 128, N = 128, K = 8 per instruction) and read
// back with tcgen05.ld for a fused epilogue.  One CTA of 4 warps per tile:
// warp 0 lane 0 issues the TMA loads, warp 1 lane 0 issues the MMAs, all four
// warps drain the accumulator (warp w owns TMEM lanes 32w .. 32w + 31).
//
// Use: the Newton-Schulz refinement of W (mixed precision): C = W R, computed
// as W Q^T with Q = R^T, lower tiles only (C is symmetric), W64 += C
// mirrored.  (The correction is small next to W, so single TF32 products
// suffice here; the factorisation and S use the split-TF32 kernel of
// cholinv_tc.cu.)  This file also packs the operands and encodes the tensor
// maps used by both kernels.
//
// Every wait on an mbarrier is bounded (SM cycles); on expiry the kernel
// records an error code, drains what it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <mutex>

#include "glasso_internal.h"
#include "tc_ptx.h"

namespace glx {
namespace {
using namespace ptx;

constexpr int TBM = 128, TBN = 128, TBK = 32, TST = 4;
constexpr uint32_t TILE_BYTES = TBM * TBK * 4;  // 16 KB, one operand tile
constexpr int TTHREADS = 128;
constexpr uint32_t TMEM_COLS = 128;

struct __align__(1024) TcSmem {
    float a[TST][TBM * TBK];
    float b[TST][TBN * TBK];
    unsigned long long full[TST];
    unsigned long long empty[TST];
    unsigned long long done;
    uint32_t tmem;
};
constexpr size_t TC_SMEM = sizeof(TcSmem) + 1024;

__device__ __forceinline__ void tri_tile(int64_t t, int64_t &I, int64_t &J) {
    int64_t i = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > t) --i;
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    I = i;
    J = t - i * (i + 1) / 2;
}

enum { EPI_NS = 0 };

// Tiles of C = P Q^T, P and Q each n_rows x K (K-major).
// EPI_NS:    lower tiles, W[i][j] += C_ij, mirrored, with W = hi + lo a
//            symmetric double-float pair (FP32 arrays, row stride ldo): hi is
//            read from inh and written to outh (another buffer: P may be inh
//            itself, read by other tiles meanwhile), lo is updated in place;
//            two-sum of hi and C, the error into lo, renormalised
template <int EPI>
__global__ void __launch_bounds__(TTHREADS, 1)
    k_tc_lower(const __grid_constant__ CUtensorMap tp, const __grid_constant__ CUtensorMap tq,
               int64_t nrows, int64_t K, const float *__restrict__ inh, float *__restrict__ outh,
               float *__restrict__ outl, int64_t ldo, int *err) {
    extern __shared__ unsigned char raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t ti, tj;
    tri_tile(blockIdx.x, ti, tj);
    const int nk = (int)((K + TBK - 1) / TBK);

    if (threadIdx.x == 0) {
        for (int s = 0; s < TST; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], 1);
        }
        mbar_init(&sm.done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sm.tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;

    int issued = 0;  // TMA stage loads issued (producer)
    if (warp == 0 && lane == 0) {
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % TST;
            if (kt >= TST && !mbar_wait(&sm.empty[s], ((kt / TST) & 1) ^ 1)) {
                atomicExch(err, 1);
                break;
            }
            mbar_expect_tx(&sm.full[s], 2 * TILE_BYTES);
            tma_2d(&sm.a[s][0], &tp, kt * TBK, (int)(ti * TBM), &sm.full[s]);
            tma_2d(&sm.b[s][0], &tq, kt * TBK, (int)(tj * TBN), &sm.full[s]);
            ++issued;
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = tf32_idesc();
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % TST;
            if (!mbar_wait(&sm.full[s], (kt / TST) & 1)) {
                atomicExch(err, 2);
                break;
            }
            tc_fence_after();
            const unsigned long long ad = sw128_desc(smem_u32(&sm.a[s][0]));
            const unsigned long long bd = sw128_desc(smem_u32(&sm.b[s][0]));
#pragma unroll
            for (int kk = 0; kk < TBK / 8; ++kk)
                umma_tf32(tmem, ad + 2ull * kk, bd + 2ull * kk, idesc, (kt | kk) != 0);
            umma_commit(&sm.empty[s]);
        }
        umma_commit(&sm.done);
    }
    __syncwarp();
    // warp-uniform outcome: the TMEM loads of the epilogue need the whole warp
    const bool ok = __all_sync(0xffffffffu, mbar_wait(&sm.done, 0));
    tc_fence_after();
    // the tile goes through the idle stage buffers (128 x 129 floats) so that
    // both the lower entries and their mirror images are updated by rows
    float(*T)[TBN + 1] = reinterpret_cast<float(*)[TBN + 1]>(&sm.a[0][0]);
    static_assert(sizeof(float) * TBM * (TBN + 1) <= sizeof(float) * 2 * TST * TBM * TBK, "staging tile");
    if (ok) {
#pragma unroll 1
        for (int cb = 0; cb < TBN / 32; ++cb) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 32), v);
#pragma unroll
            for (int c = 0; c < 32; ++c) T[warp * 32 + lane][cb * 32 + c] = v[c];
        }
    } else if (lane == 0) {
        atomicExch(err, 3);
    }
    const int allok = __syncthreads_and(ok);
    // (h, l) + x for the double-float W = hi + lo: two-sum of h and x, the
    // error into l, renormalised.  Four rows of a warp's share at a time, all
    // loads issued before the stores (one round trip per group).
    float *__restrict__ oh = outh;
    float *__restrict__ ol = outl;
    auto dfadd = [](float h, float l, float x, float &h2, float &l3) {
        const float sm = __fadd_rn(h, x), bb = __fsub_rn(sm, h);
        const float er = __fadd_rn(__fsub_rn(h, __fsub_rn(sm, bb)), __fsub_rn(x, bb));
        const float l2 = __fadd_rn(l, er);
        h2 = __fadd_rn(sm, l2);
        l3 = __fsub_rn(l2, __fsub_rn(h2, sm));
    };
    constexpr int RG = 4, NW = TTHREADS / 32;
    if (allok) {
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            // pass 0: entries (i, j), j <= i, by rows i (lanes along j);
            // pass 1: their mirror images (j, i), j < i, by rows j (lanes
            // along i) -- W is kept symmetric, so (j, i) holds the same pair
            // as (i, j) and gets the same sum
#pragma unroll 1
            for (int r0 = warp * RG; r0 < TBM; r0 += NW * RG) {
                int64_t at[RG][4];
                bool act[RG][4];
                float h[RG][4], l[RG][4], x[RG][4];
#pragma unroll
                for (int u = 0; u < RG; ++u)
#pragma unroll
                    for (int cb = 0; cb < 4; ++cb) {
                        const int a = r0 + u, b = cb * 32 + lane;  // a: the row's tile index
                        int64_t i, j;
                        if (pass == 0) {
                            i = ti * TBM + a;
                            j = tj * TBN + b;
                            act[u][cb] = i < nrows && j < nrows && j <= i;
                            at[u][cb] = i * ldo + j;
                            x[u][cb] = T[a][b];
                        } else {
                            j = tj * TBN + a;
                            i = ti * TBM + b;
                            act[u][cb] = i < nrows && j < nrows && j < i;
                            at[u][cb] = j * ldo + i;
                            x[u][cb] = T[b][a];
                        }
                        h[u][cb] = act[u][cb] ? inh[at[u][cb]] : 0.f;
                        l[u][cb] = act[u][cb] ? ol[at[u][cb]] : 0.f;
                    }
#pragma unroll
                for (int u = 0; u < RG; ++u)
#pragma unroll
                    for (int cb = 0; cb < 4; ++cb)
                        if (act[u][cb]) {
                            float h2, l3;
                            dfadd(h[u][cb], l[u][cb], x[u][cb], h2, l3);
                            oh[at[u][cb]] = h2;
                            ol[at[u][cb]] = l3;
                        }
            }
        }
    }
    // error path: wait (bounded) for the producer's copies still in flight;
    // only the last TST issued stages can be outstanding
    if (warp == 0 && lane == 0 && !ok) {
        for (int kt = issued > TST ? issued - TST : 0; kt < issued; ++kt)
            mbar_wait(&sm.full[kt % TST], (kt / TST) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
}

// ---- operand packing -----------------------------------------------------
// Qp[j][k] = R[k][j] for j, k < n, zero in the padding (ld = ldp).
__global__ void k_transpose_pad(const float *__restrict__ R, int64_t n, float *__restrict__ Qp,
                                int64_t ldp) {
    __shared__ float t[32][33];
    const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t k = by + r, j = bx + threadIdx.x;
        t[r][threadIdx.x] = (k < n && j < n) ? R[k * n + j] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t j = bx + r, k = by + threadIdx.x;
        if (j < ldp && k < ldp) Qp[j * ldp + k] = t[threadIdx.x][r];
    }
}

// Up[i][k] = U[i][k] (FP32), zero padding.
__global__ void k_copy_pad(const float *__restrict__ U, int64_t n, float *__restrict__ Up, int64_t ldp) {
    const int64_t i = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t row = i + r, col = k0 + threadIdx.x;
        if (row < ldp && col < ldp) Up[row * ldp + col] = (row < n && col < n) ? U[row * n + col] : 0.f;
    }
}

// Wp[i][k] = W[i][k] (FP32), zero padding.
__global__ void k_pack_w(const float *__restrict__ W, int64_t n, float *__restrict__ Wp, int64_t ldp) {
    const int64_t total = ldp * ldp;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / ldp, k = t % ldp;
        Wp[t] = (i < n && k < n) ? W[i * n + k] : 0.f;
    }
}

// Xt[i][k] = X[k][i] - mu_i as FP32 (i < n, k < m), zero padding (ld = ldp).
template <typename TIN>
__global__ void k_xt_pad(const TIN *__restrict__ X, int64_t m, int64_t n, const double *__restrict__ mu,
                         float *__restrict__ Xt, int64_t ldp) {
    __shared__ float t[32][33];
    const int64_t bk = (int64_t)blockIdx.x * 32, bi = (int64_t)blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t k = bk + r, i = bi + threadIdx.x;
        float v = 0.f;
        if (k < m && i < n) v = (float)((double)X[k * n + i] - (mu ? mu[i] : 0.0));
        t[r][threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int64_t i = bi + r, k = bk + threadIdx.x;
        if (i < n && k < ldp) Xt[i * ldp + k] = t[threadIdx.x][r];
    }
}

// ---- host: tensor maps -----------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

cudaError_t get_encode() {
    std::lock_guard<std::mutex> lk(g_encode_mu);
    if (g_encode) return cudaSuccess;
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return cudaSuccess;
}

// 2-D FP32 map over `rows` x `cols` (cols contiguous, row stride ld floats),
// box 32 x 128 with 128-byte swizzle.
cudaError_t make_map(CUtensorMap *map, const float *base, int64_t rows, int64_t cols, int64_t ld) {
    cudaError_t e = get_encode();
    if (e != cudaSuccess) return e;
    if (((uintptr_t)base & 15) || ((ld * 4) & 15)) return cudaErrorInvalidValue;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
    cuuint32_t box[2] = {TBK, TBM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)base, dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

OncePerDevice g_tc_once[1];

// P: nrows x kp (row stride ldp_), Q: nrows x K (row stride ld); the k-loop
// runs to K, and TMA fills P's columns beyond kp with zeros.
template <int EPI>
cudaError_t launch_lower(const float *P, int64_t kp, int64_t ldp_, const float *Q, int64_t nrows,
                         int64_t K, int64_t ld, const float *inh, float *outh, float *outl, int64_t ldo,
                         int *err, cudaStream_t st) {
    int dev = 0;
    cudaError_t ie = g_tc_once[EPI].run(dev, [](int) {
        return cudaFuncSetAttribute(k_tc_lower<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    });
    if (ie != cudaSuccess) return ie;
    CUtensorMap mp, mq;
    cudaError_t e = make_map(&mp, P, nrows, kp, ldp_);
    if (e != cudaSuccess) return e;
    e = make_map(&mq, Q, nrows, K, ld);
    if (e != cudaSuccess) return e;
    const int64_t nt = (nrows + TBM - 1) / TBM;
    k_tc_lower<EPI><<<(unsigned)(nt * (nt + 1) / 2), TTHREADS, TC_SMEM, st>>>(mp, mq, nrows, K, inh,
                                                                            outh, outl, ldo, err);
    counted(1);
    return cudaGetLastError();
}

inline unsigned gridn(int64_t work, int per = 256) {
    int64_t g = (work + per - 1) / per;
    return (unsigned)lmax(1, lmin(g, 152 * 16));
}

}  // namespace

int64_t tc_pad(int64_t n) { return (n + 31) / 32 * 32; }

cudaError_t make_tmap(CUtensorMap *map, const float *base, int64_t rows, int64_t cols, int64_t ld) {
    return make_map(map, base, rows, cols, ld);
}

// W += W R (lower tiles, mirrored) for the double-float W = hi + lo
// (symmetric, row stride n): hi is read from Whi and the new hi written to
// Whi_next (a different buffer), lo is updated in place.  The product takes
// hi and R32 (row-major, ld n) as TF32 operands; hi is read in place when its
// rows are 16-byte multiples (n % 4 == 0), else through the padded copy Wp.
// Qp (and Wp) are scratch of tc_pad(n)^2 floats.
cudaError_t ns_gemm_tc(const float *Whi, float *Whi_next, float *Wlo, const float *R32, int64_t n,
                       float *Wp, float *Qp, int *err, cudaStream_t st) {
    const int64_t ldp = tc_pad(n);
    const dim3 tg((unsigned)(ldp / 32), (unsigned)(ldp / 32)), tb(32, 8);
    k_transpose_pad<<<tg, tb, 0, st>>>(R32, n, Qp, ldp);
    counted(1);
    if (n % 4 == 0)
        return launch_lower<EPI_NS>(Whi, n, n, Qp, n, ldp, ldp, Whi, Whi_next, Wlo, n, err, st);
    k_pack_w<<<gridn(ldp * ldp), 256, 0, st>>>(Whi, n, Wp, ldp);
    counted(1);
    return launch_lower<EPI_NS>(Wp, ldp, ldp, Qp, n, ldp, ldp, Whi, Whi_next, Wlo, n, err, st);
}

// Up = U padded (ld = tc_pad(n)), Ut = U^T padded.
cudaError_t pad_and_transpose(const float *U, int64_t n, float *Up, float *Ut, cudaStream_t st) {
    const int64_t ldp = tc_pad(n);
    const dim3 tg((unsigned)(ldp / 32), (unsigned)(ldp / 32)), tb(32, 8);
    k_transpose_pad<<<tg, tb, 0, st>>>(U, n, Ut, ldp);
    k_copy_pad<<<tg, tb, 0, st>>>(U, n, Up, ldp);
    counted(2);
    return cudaGetLastError();
}

// S = (X - mu)^T (X - mu) / m from X (m x n, FP32 or FP64 values rounded to
// FP32) on the tensor cores, split TF32 with unbiased summation; Xt is
// scratch of n x tc_pad(m) floats.
cudaError_t syrk_tc(const void *X, int dtype, int64_t m, int64_t n, const double *mu, double *S,
                    float *Xt, int *err, cudaStream_t st) {
    const int64_t ldp = tc_pad(m);
    const dim3 tg((unsigned)(ldp / 32), (unsigned)((n + 31) / 32)), tb(32, 8);
    if (dtype == GLASSO_F32)
        k_xt_pad<float><<<tg, tb, 0, st>>>((const float *)X, m, n, mu, Xt, ldp);
    else
        k_xt_pad<double><<<tg, tb, 0, st>>>((const double *)X, m, n, mu, Xt, ldp);
    counted(1);
    return syrk_split(Xt, n, m, ldp, 1.0 / (double)m, S, err, st);
}

}  // namespace glx
