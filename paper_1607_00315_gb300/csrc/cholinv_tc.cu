// FP32 Cholesky factorisation with the inverse of its factor, and
// W = A^{-1} = X^T X with X = L^{-1}, for the mixed-precision solve: the
// factorisation gives the positive-definiteness test and log det A of the
// line search (Section 6.1.2), W is eq. gradHes.  Every O(n^3) contraction
// runs on the tcgen05 tensor cores as a split-TF32 product: each operand
// value x = hi + lo with hi the TF32 rounding of x and lo = x - hi (exact in
// FP32), and C = P_hi Q_hi + P_hi Q_lo + P_lo Q_hi, which keeps about 2^-21
// relative accuracy per product where a single TF32 product keeps 2^-11.
//
// Recursive form, node [o, o + s) split at o + s1 (s1 a multiple of 128):
//   [L11, X11] = node(A11)
//   L21 = A21 X11^T                  panel, into scratch Z21
//   A22 -= L21 L21^T                 lower tiles, in place
//   [L22, X22] = node(A22)
//   Yt  = Xt11 L21^T  (= (L21 X11)^T) into scratch Z12
//   X21 = -X22 Yt^T, and Xt12 = X21^T
// A node of at most 32 tiles (s <= 4096; the caller may lower the bound or
// ask for the plain recursion) is instead factored and inverted by one
// persistent task-graph launch (chol_dag.cu).
// Leaves (s <= 128) are factored and inverted by one CTA in shared memory
// (FP32), which also records the FP64 diagonal of L for log det A.  Per
// output tile the k range skips the zero triangles of X and Xt = X^T.
//
// GEMM kernel: one CTA per 128 x 128 output tile; warp 0 issues TMA loads of
// 128 x 32 FP32 tiles (128-byte swizzle) into a 3-stage ring, warps 2-5 split
// each landed tile into hi and lo tiles in shared memory (same swizzled
// positions), warp 1 issues three tcgen05.mma.kind::tf32 per 8-wide k step
// into TMEM, and warps 6-13 drain TMEM into FP32 registers and the epilogue
// (see k_tcx on how the sums are kept unbiased).  Every mbarrier wait is
// bounded; on expiry the kernel records a code, lets its own copies land,
// frees TMEM and returns.
#include <cuda.h>
#include <math.h>

#include "glasso_internal.h"
#include "tc_ptx.h"

namespace glx {
namespace {
using namespace ptx;

constexpr int XM = 128, XN = 128, XK = 32, XST = 3, XNB = 3;
constexpr int XTHREADS = 448;
constexpr uint32_t XTILE = XM * XK * 4;  // 16 KB

struct __align__(1024) XSmem {
    float a[XST][XM * XK];
    float b[XST][XN * XK];
    float alo[XST][XM * XK];
    float blo[XST][XN * XK];
    unsigned long long full[XST], conv[XST], empty[XST], done;
    unsigned long long mfull[XNB], mfree[XNB];
    uint32_t tmem;
};
constexpr size_t XSMEM = sizeof(XSmem) + 1024;

enum { XE_ASSIGN = 0, XE_SUB = 1, XE_SYM = 2, XE_SYM64 = 3 };

struct XArgs {
    int64_t M, N, K;        // output rows (rows of P), output columns (rows of Q), depth
    int tiles_n;            // tile columns of a full grid
    int lower;              // only tiles ti >= tj (triangular enumeration)
    int kbeg_i, kend_i, kend_j;  // per-tile k range: [ti*128, .), [., (ti+1)*128), [., (tj+1)*128)
    int drain;              // sum the main products outside the tensor core (see k_tcx)
    int epi;                // XE_ASSIGN: out = alpha C (+ outT = its transpose)
                            // XE_SUB:    out -= C on j <= i
                            // XE_SYM:    out[i][j] = out[j][i] = C on j <= i
                            // XE_SYM64:  out64[i][j] = out64[j][i] = scale C on j <= i (FP64)
    float alpha;
    double scale;
    double *out64;
    float *out;
    int64_t ldo;
    float *outT;
    int64_t ldt;
    const int *info;        // skip the tile when *info != 0 (a failed pivot upstream)
    int *err;
};

__device__ __forceinline__ void tri_tile_x(int64_t t, int64_t &I, int64_t &J) {
    int64_t i = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > t) --i;
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    I = i;
    J = t - i * (i + 1) / 2;
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

// Roles: warp 0 TMA producer, warp 1 MMA issuer, warps 2-5 split the landed
// tiles, warps 6-13 drain TMEM: warp w reads TMEM lanes 32 (w % 4) .. (the
// rows it may access) and columns 64 ((w - 6) / 4) .. + 63.
//
// Accumulation.  The tensor core sums each 8-wide k step into its FP32
// accumulator with a truncation (measured on this GPU: a bias of about one
// FP32 ulp of the accumulator per step, toward zero), which over a long k
// range becomes a systematic relative error of (k / 8) 2^-24 -- harmless for
// the inverse (refined afterwards) but not for a log-determinant summed over
// n pivots.  With `drain`, the main product hi hi of every pair of 8-wide
// steps goes to a fresh TMEM buffer (three in rotation) that the drain warps
// add into FP32 registers with round-to-nearest (measured bias: about one
// ulp of each 16-wide partial, independent of k); the small hi lo + lo hi
// terms keep one TMEM accumulator.  Without it, all products accumulate in
// TMEM.
__global__ void __launch_bounds__(XTHREADS, 1)
    k_tcx(const __grid_constant__ CUtensorMap tp, const __grid_constant__ CUtensorMap tq,
          const XArgs a) {
    extern __shared__ unsigned char raw[];
    XSmem &sm = *reinterpret_cast<XSmem *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t ti, tj;
    if (a.lower) {
        tri_tile_x(blockIdx.x, ti, tj);
    } else {
        ti = blockIdx.x / a.tiles_n;
        tj = blockIdx.x % a.tiles_n;
    }
    int64_t kb = 0, ke = a.K;
    if (a.kbeg_i) kb = lmax(kb, ti * XM);
    if (a.kend_i) ke = lmin(ke, (ti + 1) * XM);
    if (a.kend_j) ke = lmin(ke, (tj + 1) * XN);
    const int nk = ke > kb ? (int)((ke - kb + XK - 1) / XK) : 0;
    const bool drain = a.drain != 0;
    const uint32_t ncols = drain ? 512u : 128u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < XST; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.conv[s], 4);
            mbar_init(&sm.empty[s], 1);
        }
        for (int b = 0; b < XNB; ++b) {
            mbar_init(&sm.mfull[b], 1);
            mbar_init(&sm.mfree[b], 8);
        }
        mbar_init(&sm.done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sm.tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;  // column 0: the accumulator (drain: the hi lo + lo hi terms)
    // inputs come from the preceding kernel from here on
    pdl_wait();
    pdl_trigger();
    if (a.info && *a.info != 0) {  // an earlier pivot failed: nothing to do (same in every thread)
        tc_fence_before();
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                         : "memory");
        return;
    }
    const int lw = warp & 3;
    const uint32_t lane_off = (uint32_t)(lw * 32) << 16;

    int issued = 0;
    bool ok = true;
    if (warp >= 6) {
        // drain warps: half a row of C, summed in FP32, then the epilogue
        constexpr int HC = XN / 2;
        const uint32_t col0 = (uint32_t)(((warp - 6) >> 2) * HC);
        float acc[HC];
#pragma unroll
        for (int c = 0; c < HC; ++c) acc[c] = 0.f;
        if (nk > 0) {
            if (drain) {
                // add the main product of every pair of 8-wide steps (round to nearest)
                const int npairs = nk * (XK / 16);
                for (int pr = 0; pr < npairs; ++pr) {
                    const int b = pr % XNB;
                    // warp-uniform outcome: the TMEM loads below need the whole warp
                    const bool got = __all_sync(0xffffffffu, mbar_wait(&sm.mfull[b], (pr / XNB) & 1));
                    if (!got) {
                        if (lane == 0) atomicExch(a.err, 16);
                        break;
                    }
                    tc_fence_after();
                    uint32_t v0[32], v1[32];
                    tmem_ld32_issue(tmem + lane_off + 128u * (uint32_t)(b + 1) + col0, v0);
                    tmem_ld32_issue(tmem + lane_off + 128u * (uint32_t)(b + 1) + col0 + 32u, v1);
                    tmem_wait_ld();
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        acc[c] += __uint_as_float(v0[c]);
                        acc[32 + c] += __uint_as_float(v1[c]);
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sm.mfree[b]);
                }
            }
            __syncwarp();
            ok = __all_sync(0xffffffffu, mbar_wait(&sm.done, 0));
            tc_fence_after();
            if (!ok && lane == 0) atomicExch(a.err, 14);
        }
        // stage C in the (now idle) stage buffers, padded rows, then write it out
        // with coalesced rows (and, for outT / the mirror, columns); every drain
        // warp reaches the named barrier, whatever its wait returned
        float(*Ct)[XM + 1] = reinterpret_cast<float(*)[XM + 1]>(&sm.a[0][0]);
        if (ok) {
            const int rl = lw * 32 + lane;
#pragma unroll
            for (int cb = 0; cb < HC / 32; ++cb) {
                float v[32];
                if (nk > 0) {
                    tmem_ld32(tmem + lane_off + col0 + (uint32_t)(cb * 32), v);
                } else {
#pragma unroll
                    for (int c = 0; c < 32; ++c) v[c] = 0.f;
                }
#pragma unroll
                for (int c = 0; c < 32; ++c) Ct[rl][col0 + cb * 32 + c] = acc[cb * 32 + c] + v[c];
            }
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");
        if (ok) {
            const int et = threadIdx.x - 192, wr = et >> 5;  // 8 warps x 32 lanes
            if (a.epi == XE_SUB) {
                // read-modify-write: the loads of four rows are issued before
                // their stores (one round trip per group, not per element)
                float *__restrict__ o = a.out;
#pragma unroll 1
                for (int r0 = wr * 4; r0 < XM; r0 += 32) {
                    float cur[4][XN / 32];
                    bool act[4][XN / 32];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int p = 0; p < XN / 32; ++p) {
                            const int64_t i = ti * XM + r0 + u, j = tj * XN + lane + 32 * p;
                            act[u][p] = i < a.M && j < a.N && j <= i;
                            cur[u][p] = act[u][p] ? o[i * a.ldo + j] : 0.f;
                        }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int p = 0; p < XN / 32; ++p)
                            if (act[u][p]) {
                                const int64_t i = ti * XM + r0 + u, j = tj * XN + lane + 32 * p;
                                o[i * a.ldo + j] = cur[u][p] - Ct[r0 + u][lane + 32 * p];
                            }
                }
            } else {
#pragma unroll 1
                for (int r = wr; r < XM; r += 8) {
                    const int64_t i = ti * XM + r;
                    if (i >= a.M) break;
#pragma unroll
                    for (int p = 0; p < XN / 32; ++p) {
                        const int cc = lane + 32 * p;
                        const int64_t j = tj * XN + cc;
                        if (j >= a.N) continue;
                        const float v = Ct[r][cc];
                        if (a.epi == XE_ASSIGN) a.out[i * a.ldo + j] = a.alpha * v;
                        else if (j <= i) {
                            if (a.epi == XE_SYM) a.out[i * a.ldo + j] = v;
                            else a.out64[i * a.ldo + j] = a.scale * (double)v;
                        }
                    }
                }
            }
            if (a.outT || a.epi == XE_SYM || a.epi == XE_SYM64) {
#pragma unroll 1
                for (int cc = wr; cc < XN; cc += 8) {
                    const int64_t j = tj * XN + cc;
                    if (j >= a.N) break;
#pragma unroll
                    for (int p = 0; p < XM / 32; ++p) {
                        const int r = lane + 32 * p;
                        const int64_t i = ti * XM + r;
                        if (i >= a.M) continue;
                        const float v = Ct[r][cc];
                        if (a.epi == XE_ASSIGN) a.outT[j * a.ldt + i] = a.alpha * v;
                        else if (j < i) {
                            if (a.epi == XE_SYM) a.out[j * a.ldo + i] = v;
                            else a.out64[j * a.ldo + i] = a.scale * (double)v;
                        }
                    }
                }
            }
        }
    } else if (nk > 0) {
        if (warp == 0 && lane == 0) {
            for (int kt = 0; kt < nk; ++kt) {
                const int s = kt % XST;
                if (kt >= XST && !mbar_wait(&sm.empty[s], ((kt / XST) & 1) ^ 1)) {
                    atomicExch(a.err, 11);
                    break;
                }
                mbar_expect_tx(&sm.full[s], 2 * XTILE);
                const int x = (int)(kb + (int64_t)kt * XK);
                tma_2d(&sm.a[s][0], &tp, x, (int)(ti * XM), &sm.full[s]);
                tma_2d(&sm.b[s][0], &tq, x, (int)(tj * XN), &sm.full[s]);
                ++issued;
            }
        } else if (warp == 1 && lane == 0) {
            const uint32_t idesc = tf32_idesc(XM, XN);
            bool mok = true;
            for (int kt = 0; kt < nk && mok; ++kt) {
                const int s = kt % XST;
                if (!mbar_wait(&sm.conv[s], (kt / XST) & 1)) {
                    atomicExch(a.err, 12);
                    break;
                }
                tc_fence_after();
                const unsigned long long ah = sw128_desc(smem_u32(&sm.a[s][0]));
                const unsigned long long bh = sw128_desc(smem_u32(&sm.b[s][0]));
                const unsigned long long al = sw128_desc(smem_u32(&sm.alo[s][0]));
                const unsigned long long bl = sw128_desc(smem_u32(&sm.blo[s][0]));
#pragma unroll
                for (int kk = 0; kk < XK / 8; ++kk) {
                    const uint32_t first = (kt | kk) != 0;
                    if (drain) {
                        // pair p of 8-wide steps into buffer p % XNB
                        const int step = kt * (XK / 8) + kk, pr = step >> 1, b = pr % XNB;
                        if ((step & 1) == 0 && pr >= XNB &&
                            !mbar_wait(&sm.mfree[b], ((pr / XNB) & 1) ^ 1)) {
                            atomicExch(a.err, 15);
                            mok = false;
                            break;
                        }
                        tc_fence_after();
                        umma_tf32(tmem + 128u * (uint32_t)(b + 1), ah + 2ull * kk, bh + 2ull * kk, idesc,
                                  (uint32_t)(step & 1));
                        if (step & 1) umma_commit(&sm.mfull[b]);
                        umma_tf32(tmem, ah + 2ull * kk, bl + 2ull * kk, idesc, first);
                    } else {
                        umma_tf32(tmem, ah + 2ull * kk, bh + 2ull * kk, idesc, first);
                        umma_tf32(tmem, ah + 2ull * kk, bl + 2ull * kk, idesc, 1u);
                    }
                    umma_tf32(tmem, al + 2ull * kk, bh + 2ull * kk, idesc, 1u);
                }
                umma_commit(&sm.empty[s]);
            }
            umma_commit(&sm.done);
        } else if (warp >= 2) {
            // split each landed stage: hi in place, lo into the lo tiles
            const int ct = threadIdx.x - 64;  // 0 .. 127
            for (int kt = 0; kt < nk; ++kt) {
                const int s = kt % XST;
                if (!mbar_wait(&sm.full[s], (kt / XST) & 1)) {
                    atomicExch(a.err, 13);
                    break;
                }
                float4 *pa = reinterpret_cast<float4 *>(&sm.a[s][0]);
                float4 *pb = reinterpret_cast<float4 *>(&sm.b[s][0]);
                float4 *la = reinterpret_cast<float4 *>(&sm.alo[s][0]);
                float4 *lb = reinterpret_cast<float4 *>(&sm.blo[s][0]);
#pragma unroll
                for (int r = 0; r < (XM * XK / 4) / 128; ++r) {
                    const int q = ct + 128 * r;
                    float4 v = pa[q], h;
                    h.x = tf32_round(v.x); h.y = tf32_round(v.y);
                    h.z = tf32_round(v.z); h.w = tf32_round(v.w);
                    pa[q] = h;
                    la[q] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
                    v = pb[q];
                    h.x = tf32_round(v.x); h.y = tf32_round(v.y);
                    h.z = tf32_round(v.z); h.w = tf32_round(v.w);
                    pb[q] = h;
                    lb[q] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.conv[s]);
            }
        }
        __syncwarp();
        ok = mbar_wait(&sm.done, 0);
        tc_fence_after();
    }
    // error path: the producer waits (bounded) for its copies still in flight
    if (!ok && warp == 0 && lane == 0) {
        for (int kt = issued > XST ? issued - XST : 0; kt < issued; ++kt)
            mbar_wait(&sm.full[kt % XST], (kt / XST) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                     : "memory");
}

OncePerDevice g_tcx_once;

// C (M x N) from P (M x K) and Q (N x K), both sub-matrices of FP32 buffers
// with row stride ld (a multiple of 32 floats, 16-byte aligned bases).
cudaError_t tcx(const float *P, const float *Q, int64_t M, int64_t N, int64_t K, int64_t ld,
                bool lower, int kbeg_i, int kend_i, int kend_j, bool drain, int epi, float alpha,
                float *out, int64_t ldo, float *outT, int64_t ldt, const int *info, int *err,
                cudaStream_t st, double scale64 = 1.0) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    int dev = 0;
    cudaError_t ie = g_tcx_once.run(dev, [](int) {
        return cudaFuncSetAttribute(k_tcx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)XSMEM);
    });
    if (ie != cudaSuccess) return ie;
    CUtensorMap mp, mq;
    cudaError_t e = make_tmap(&mp, P, M, lmax(K, 1), ld);
    if (e != cudaSuccess) return e;
    e = make_tmap(&mq, Q, N, lmax(K, 1), ld);
    if (e != cudaSuccess) return e;
    XArgs a;
    a.M = M;
    a.N = N;
    a.K = K;
    const int64_t tm = (M + XM - 1) / XM, tn = (N + XN - 1) / XN;
    a.tiles_n = (int)tn;
    a.lower = lower ? 1 : 0;
    a.kbeg_i = kbeg_i;
    a.kend_i = kend_i;
    a.kend_j = kend_j;
    a.drain = drain ? 1 : 0;
    a.epi = epi;
    a.alpha = alpha;
    a.scale = 0.0;
    a.out64 = nullptr;
    a.out = out;
    a.ldo = ldo;
    a.outT = outT;
    a.ldt = ldt;
    a.info = info;
    a.err = err;
    if (epi == XE_SYM64) {
        a.out64 = reinterpret_cast<double *>(out);
        a.scale = scale64;
        a.out = nullptr;
    }
    const int64_t grid = lower ? tm * (tm + 1) / 2 : tm * tn;
    // programmatic serialisation: the prologue (barriers, TMEM) overlaps the
    // predecessor's tail; the kernel waits for it before reading inputs
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(XTHREADS);
    cfg.dynamicSmemBytes = XSMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t le = cudaLaunchKernelEx(&cfg, k_tcx, mp, mq, a);
    counted(1);
    if (le != cudaSuccess) return le;
    return cudaGetLastError();
}

struct Rec {
    float *A, *X, *Xt, *Z;
    int64_t ld;
    double *ldiag;
    DevScalars *sc;
    cudaStream_t st;
    cudaStream_t side;  // optional: Yt runs here, beside SYRK and the right subtree
    cudaEvent_t ev_a, ev_b;
    int dag_tiles;      // largest block of one task-graph launch (0: default, 1: none)
    int dag_share;      // a task-graph launch takes at most 1 / dag_share of the SMs
};

cudaError_t node(const Rec &r, int64_t o, int64_t s) {
    if (s <= 128) return chol_leaf32(r.A, r.ld, o, (int)s, r.X, r.Xt, r.ldiag, r.sc, r.st);
    // the task graph's counters use Z's diagonal block, which no enclosing
    // node's scratch (Z21 below it, Z12 beside it) overlaps
    if (r.dag_tiles != 1 && chol_dag_fits(s, r.dag_tiles))
        return chol_dag(r.A, r.ld, o, s, r.X, r.Xt, r.ldiag, reinterpret_cast<unsigned *>(r.Z + o * r.ld + o),
                        r.sc, r.st, 0, r.dag_share);
    const int64_t s1 = ((s / 2) + 127) / 128 * 128, s2 = s - s1;
    const int64_t ld = r.ld;
    int *err = &r.sc->tc_err;
    const int *info = &r.sc->info;
    cudaError_t e = node(r, o, s1);
    if (e != cudaSuccess) return e;
    float *A21 = r.A + (o + s1) * ld + o, *A22 = r.A + (o + s1) * ld + o + s1;
    float *Z21 = r.Z + (o + s1) * ld + o, *Z12 = r.Z + o * ld + o + s1;
    const float *X11 = r.X + o * ld + o, *Xt11 = r.Xt + o * ld + o;
    float *X21 = r.X + (o + s1) * ld + o, *X22 = r.X + (o + s1) * ld + o + s1;
    float *Xt12 = r.Xt + o * ld + o + s1;
    // L21 = A21 X11^T (X11 lower: k < (tj + 1) 128)
    e = tcx(A21, X11, s2, s1, s1, ld, false, 0, 0, 1, true, XE_ASSIGN, 1.f, Z21, ld, nullptr, 0, info,
            err, r.st);
    if (e != cudaSuccess) return e;
    // Yt = Xt11 L21^T (Xt11 upper: k >= ti 128).  It needs only the left
    // subtree and the panel, so with a side stream it runs beside SYRK and the
    // right subtree (it writes rows [o, o + s1) of Z; the right subtree's
    // scratch lies in rows >= o + s1)
    cudaStream_t ys = r.st;
    if (r.side) {
        e = cudaEventRecord(r.ev_a, r.st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(r.side, r.ev_a, 0);
        if (e != cudaSuccess) return e;
        ys = r.side;
    }
    e = tcx(Xt11, Z21, s1, s2, s1, ld, false, 1, 0, 0, false, XE_ASSIGN, 1.f, Z12, ld, nullptr, 0, info,
            err, ys);
    if (e != cudaSuccess) return e;
    if (r.side) {
        e = cudaEventRecord(r.ev_b, r.side);
        if (e != cudaSuccess) return e;
    }
    // A22 -= L21 L21^T
    e = tcx(Z21, Z21, s2, s2, s1, ld, true, 0, 0, 0, true, XE_SUB, 1.f, A22, ld, nullptr, 0, info, err,
            r.st);
    if (e != cudaSuccess) return e;
    e = node(r, o + s1, s2);
    if (e != cudaSuccess) return e;
    // (the last record of ev_b follows this node's Yt on the side stream)
    if (r.side) {
        e = cudaStreamWaitEvent(r.st, r.ev_b, 0);
        if (e != cudaSuccess) return e;
    }
    // X21 = -X22 Yt^T (X22 lower: k < (ti + 1) 128), Xt12 = X21^T
    return tcx(X22, Z12, s2, s1, s2, ld, false, 0, 1, 0, false, XE_ASSIGN, -1.f, X21, ld, Xt12, ld,
               info, err, r.st);
}

}  // namespace

// Factor A (n x n FP32, lower triangle, row stride ld = tc_pad(n)) and invert
// the factor: X = L^{-1} (lower) and Xt = X^T (upper), both with zero
// triangles; A is overwritten (trailing updates), Z is scratch (n x ld).
// sc->info = first failing pivot + 1 (0 if positive definite), sc->logdet =
// log det A (when info == 0), sc->tc_err = nonzero if a bounded wait expired.
cudaError_t cholinv_tc(float *A, int64_t n, int64_t ld, float *X, float *Xt, float *Z,
                       double *ldiag, DevScalars *sc, cudaStream_t st, cudaStream_t side,
                       cudaEvent_t ev_a, cudaEvent_t ev_b, int dag_tiles, int dag_share) {
    if (ld % 32 != 0 || ld < n) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(&sc->info, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (side && (!ev_a || !ev_b)) return cudaErrorInvalidValue;
    Rec r{A, X, Xt, Z, ld, ldiag, sc, st, side, ev_a, ev_b, dag_tiles, dag_share};
    path_hit(GLASSO_PATH_TC_FACTOR);
    e = node(r, 0, n);
    if (e != cudaSuccess) return e;
    return logdet_from_diag(ldiag, n, sc, st);
}

// C = P Q^T for n x n FP32 operands (row stride ld, a multiple of 32), split
// TF32 with the main products summed outside the tensor core: relative error
// about 2^-21 per product plus FP32 round-to-nearest summation of n / 8
// partial sums.  C (row stride ld) is written for rows and columns < n.
cudaError_t gemm_nt_split(const float *P, const float *Q, int64_t n, int64_t ld, float *C, int *err,
                          cudaStream_t st) {
    return tcx(P, Q, n, n, n, ld, false, 0, 0, 0, true, XE_ASSIGN, 1.f, C, ld, nullptr, 0, nullptr,
               err, st);
}

// S = scale Xt Xt^T (FP64, row stride n, mirrored) from Xt (n x m FP32, row
// stride ldx), split TF32 with unbiased summation (eq. cov_estimate: Xt holds
// the centred samples transposed, scale = 1 / m).
cudaError_t syrk_split(const float *Xt, int64_t n, int64_t m, int64_t ldx, double scale, double *S,
                       int *err, cudaStream_t st) {
    return tcx(Xt, Xt, n, n, m, ldx, true, 0, 0, 0, true, XE_SYM64, 1.f,
               reinterpret_cast<float *>(S), n, nullptr, 0, nullptr, err, st, scale);
}

// W = Xt Xt^T (= X^T X = A^{-1}), lower tiles mirrored, W row stride ldw.
cudaError_t lauum_tc(const float *Xt, int64_t n, int64_t ld, float *W, int64_t ldw, DevScalars *sc,
                     cudaStream_t st) {
    return tcx(Xt, Xt, n, n, n, ld, true, 1, 0, 0, false, XE_SYM, 1.f, W, ldw, nullptr, 0, &sc->info,
               &sc->tc_err, st);
}

}  // namespace glx
