// The FP32 leaf of the tensor-core factorisation (Section 6.1.2 needs the
// factorisation for the positive-definiteness test and log det A; W = A^{-1}
// of eq. gradHes follows from the inverse factor): shared by the one-CTA
// leaf kernel and the persistent tiled factorisation.
//
// One CTA of LT = 448 threads factors the diagonal block [o, o + s), s <= 128,
// of A (row stride ld) in shared memory and inverts its factor:
//  * warps 0-7 factor in 8-wide steps (right-looking): the next 8 x 8
//    diagonal block is factored by one thread of warp 0 while warps 1-7
//    apply the trailing update (look-ahead); then two threads per row form
//    the panel L_rb = A_rb X_bb^T from the block's inverse X_bb;
//  * warps 8-13 form X = L^{-1} alongside, right-looking on L X = I by block
//    rows: X_i = -X_ii sum_{j < i} L_ij X_j, each product L_ij X_j added as
//    soon as the panel of step j is final.
// (Measured variants: spreading the 8 x 8 block over eight lanes, or a
// separate doubling inverse after the factorisation, were slower.)
// Rows beyond s are identity.  leaf_factor writes the s x s block of X
// (lower, zeros above) and the FP64 diagonal of L into ldiag[o ..];
// leaf_store_xt then writes Xt = X^T (upper, zeros below).
#pragma once
#include <stdint.h>

namespace glx {
namespace leaf {

constexpr int LB = 128, LP = LB + 4;  // rows padded to 16-byte multiples
constexpr int LT = 448;               // threads of the leaf
constexpr int LF = 256;               // the factorisation's threads (warps 0-7)
constexpr size_t LEAF_SMEM = (2 * LB + 8) * LP * sizeof(float);  // L, X and the panel transposed

// Shared state of one leaf (the caller's shared memory).
struct LeafShared {
    int fail;   // first failing pivot + 1 (local index), or 0 (written by warps 0-7 only)
    int prog;   // steps of the factorisation whose panels are final (written by warps 0-7)
    int ifail;  // the inverse warps' bounded wait expired (written by them only)
};

// 1/sqrt(d) for d > 0: the hardware estimate and one Newton step
// r <- r (3 - d r^2) / 2.
__device__ __forceinline__ float rsqrt_f32(float d) {
    float r = rsqrtf(d);
    return r * fmaf(-0.5f * d * r, r, 1.5f);
}

// Named barriers of the two roles (the CTA-wide barrier is __syncthreads).
__device__ __forceinline__ void bar_factor() { asm volatile("bar.sync 2, 256;" ::: "memory"); }
__device__ __forceinline__ void bar_inverse() { asm volatile("bar.sync 3, 192;" ::: "memory"); }
// The inverse role's barrier with an OR of v over its threads: every thread
// gets the same answer, so they leave their loop together.
__device__ __forceinline__ bool bar_inverse_any(bool v) {
    unsigned r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 3, 192, p;\n"
        " selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((unsigned)v)
        : "memory");
    return r != 0;
}

// One thread: Cholesky of the 8 x 8 lower block a (registers) in place;
// rd[i] = 1 / L_ii.  Returns 0 or the failing pivot + 1.
__device__ __forceinline__ int thread_chol8(float (&a)[8][8], float (&rd)[8]) {
    int fail = 0;  // recorded, not branched on: the pivot chain stays straight-line
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float d = a[j][j];
        if (fail == 0 && !(d > 0.f)) fail = j + 1;
        d = d > 0.f ? d : 1.f;
        const float r = rsqrt_f32(d);
        rd[j] = r;
        a[j][j] = d * r;
#pragma unroll
        for (int i = j + 1; i < 8; ++i) a[i][j] *= r;
#pragma unroll
        for (int i = j + 1; i < 8; ++i)
#pragma unroll
            for (int k = j + 1; k <= i; ++k) a[i][k] = fmaf(-a[i][j], a[k][j], a[i][k]);
    }
    return fail;
}

// One thread: factor the 8 x 8 diagonal block at d of L in place and write
// its inverse into X's block (zeros above the diagonal): the eight columns of
// the inverse, x_i = (delta_ic - sum_{t < i} L_it x_t) / L_ii, are independent
// chains, so one thread keeps them all in flight.  (Spreading the columns
// over eight lanes measured about three times slower on this GPU.)  Returns
// 0 or the failing pivot + 1.
__device__ __forceinline__ int diag8(float (*L)[LP], float (*X)[LP], int d) {
    float a[8][8], x[8][8], rd[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) a[i][j] = (j <= i) ? L[d + i][d + j] : 0.f;
    const int f = thread_chol8(a, rd);
    if (f) return f;
#pragma unroll
    for (int cc = 0; cc < 8; ++cc)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i < cc) {
                x[i][cc] = 0.f;
            } else {
                float acc = (i == cc) ? 1.f : 0.f;
#pragma unroll
                for (int t = cc; t < i; ++t) acc = fmaf(-a[i][t], x[t][cc], acc);
                x[i][cc] = acc * rd[i];
            }
        }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (j <= i) L[d + i][d + j] = a[i][j];
            X[d + i][d + j] = x[i][j];
        }
    return 0;
}

__device__ __forceinline__ float dot8(float4 p0, float4 p1, float4 q0, float4 q1) {
    float a0 = p0.x * q0.x, a1 = p0.y * q0.y;
    a0 = fmaf(p0.z, q0.z, a0);
    a1 = fmaf(p0.w, q0.w, a1);
    a0 = fmaf(p1.x, q1.x, a0);
    a1 = fmaf(p1.y, q1.y, a1);
    a0 = fmaf(p1.z, q1.z, a0);
    a1 = fmaf(p1.w, q1.w, a1);
    return a0 + a1;
}

// The leaf on all LT threads of the calling CTA (every thread must call it).
// lsm: LEAF_SMEM bytes of shared memory.  A is read through L2 (it may have
// been written by other CTAs of the same launch).  Writes X's block and
// ldiag; returns 0, the failing pivot + 1 (local index), or -1 if the inverse
// warps' bounded poll of the factorisation's progress (wait_cycles) expired --
// the same in every thread; nothing is written unless it returns 0.
__device__ __forceinline__ int leaf_factor(const float *__restrict__ A, int64_t ld, int64_t o, int s,
                                           float *__restrict__ Xo, double *__restrict__ ldiag, float *lsm,
                                           LeafShared *sh, long long wait_cycles) {
    float(*L)[LP] = reinterpret_cast<float(*)[LP]>(lsm);
    float(*X)[LP] = reinterpret_cast<float(*)[LP]>(lsm + LB * LP);
    // the current panel transposed, Pt[c][r] = L[r][d0 + c]: the trailing
    // update reads four consecutive rows of a column as one 16-byte word (rows
    // four apart in L would fall on two bank groups only)
    float(*Pt)[LP] = reinterpret_cast<float(*)[LP]>(lsm + 2 * LB * LP);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // 16-byte loads of the rows (the block starts at a multiple of 128 in a
    // matrix whose row stride is a multiple of 32 floats), all issued before
    // the first shared-memory store; X starts at zero
    {
        constexpr int NQ = (LB * LB / 4 + LT - 1) / LT;
        float4 v[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int idx = tid + LT * q, r = idx / (LB / 4), c4 = 4 * (idx % (LB / 4));
            v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (idx < LB * LB / 4 && r < s && c4 <= r) {
                const float *src = A + (o + r) * ld + o + c4;
                if (c4 + 3 < s) {
                    v[q] = __ldcg(reinterpret_cast<const float4 *>(src));
                } else {
                    v[q].x = __ldcg(src);
                    if (c4 + 1 < s) v[q].y = __ldcg(src + 1);
                    if (c4 + 2 < s) v[q].z = __ldcg(src + 2);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int idx = tid + LT * q, r = idx / (LB / 4), c4 = 4 * (idx % (LB / 4));
            if (idx >= LB * LB / 4) break;
            const float e[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
            float f[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int cc = c4 + k;
                f[k] = (cc <= r && r < s) ? e[k] : (r == cc ? 1.f : 0.f);
            }
            *reinterpret_cast<float4 *>(&L[r][c4]) = make_float4(f[0], f[1], f[2], f[3]);
            *reinterpret_cast<float4 *>(&X[r][c4]) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    if (tid == 0) {
        sh->fail = 0;
        sh->prog = 0;
        sh->ifail = 0;
    }
    __syncthreads();
    if (tid < LF) {
        // ---- factorisation (warps 0-7)
        if (tid == 0) sh->fail = diag8(L, X, 0);
        bar_factor();
        for (int d0 = 0; d0 < LB - 8; d0 += 8) {
            if (*(volatile int *)&sh->fail) break;
            const int b0 = d0 + 8, R = LB - b0;  // rows below the diagonal block
            // panel: L[r][d0 + c] = sum_b L[r][d0 + b] X[d0 + c][d0 + b] (X's
            // diagonal block is zero above its diagonal); row r by the lane pair
            // (2j, 2j + 1) of a warp, four columns each: both read the row
            // before either writes it (a warp barrier, not a CTA one)
            {
                const int r = b0 + (tid >> 1), h = 4 * (tid & 1);
                float o4[4];
                if (r < LB) {
                    const float4 p0 = *reinterpret_cast<const float4 *>(&L[r][d0]);
                    const float4 p1 = *reinterpret_cast<const float4 *>(&L[r][d0 + 4]);
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        o4[c] = dot8(p0, p1, *reinterpret_cast<const float4 *>(&X[d0 + h + c][d0]),
                                     *reinterpret_cast<const float4 *>(&X[d0 + h + c][d0 + 4]));
                }
                __syncwarp();
                if (r < LB) {
                    *reinterpret_cast<float4 *>(&L[r][d0 + h]) = make_float4(o4[0], o4[1], o4[2], o4[3]);
#pragma unroll
                    for (int c = 0; c < 4; ++c) Pt[h + c][r] = o4[c];
                }
            }
            bar_factor();
            // the panel of step d0 / 8 is final (and X's diagonal block d0 / 8
            // since the step before): the inverse warps may apply it
            if (tid == 0) {
                __threadfence_block();
                *(volatile int *)&sh->prog = d0 / 8 + 1;
            }
            if (warp == 0) {
                // look-ahead: warp 0 updates the next diagonal block (36
                // entries) and one lane factors it while warps 1-7 update the
                // rest
                int ii[2], jj[2];
                float4 a0[2], a1[2], q0[2], q1[2];
                float cur[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int e = lane + 32 * u < 36 ? lane + 32 * u : 0;
                    int i = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);  // row of entry e (j <= i)
                    if ((i + 1) * (i + 2) / 2 <= e) ++i;
                    if (i * (i + 1) / 2 > e) --i;
                    ii[u] = i;
                    jj[u] = e - i * (i + 1) / 2;
                    a0[u] = *reinterpret_cast<const float4 *>(&L[b0 + i][d0]);
                    a1[u] = *reinterpret_cast<const float4 *>(&L[b0 + i][d0 + 4]);
                    q0[u] = *reinterpret_cast<const float4 *>(&L[b0 + jj[u]][d0]);
                    q1[u] = *reinterpret_cast<const float4 *>(&L[b0 + jj[u]][d0 + 4]);
                    cur[u] = L[b0 + i][b0 + jj[u]];
                }
#pragma unroll
                for (int u = 0; u < 2; ++u)
                    if (lane + 32 * u < 36) L[b0 + ii[u]][b0 + jj[u]] = cur[u] - dot8(a0[u], a1[u], q0[u], q1[u]);
                __syncwarp();
                if (lane == 0) {
                    const int f = diag8(L, X, b0);
                    if (f) sh->fail = b0 + f;
                }
            } else {
                // trailing update of the lower part outside the next diagonal
                // block, 4 x 4 register tiles (I, J), J <= I, in units of 4
                // from b0; tiles 0..2 (the next diagonal block) are warp 0's
                const int TI = R / 4, ntl = TI * (TI + 1) / 2;
                for (int qq = 3 + (tid - 32); qq < ntl; qq += LF - 32) {
                    int I = (int)((sqrtf(8.f * qq + 1.f) - 1.f) * 0.5f);
                    if ((I + 1) * (I + 2) / 2 <= qq) ++I;
                    if (I * (I + 1) / 2 > qq) --I;
                    const int J = qq - I * (I + 1) / 2;
                    const int i0 = b0 + 4 * I, j0 = b0 + 4 * J;
                    float4 pc[8], rc[8], cv[4];  // pc[c] = rows i0 .. i0 + 3 of panel column c
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        pc[c] = *reinterpret_cast<const float4 *>(&Pt[c][i0]);
                        rc[c] = *reinterpret_cast<const float4 *>(&Pt[c][j0]);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) cv[u] = *reinterpret_cast<const float4 *>(&L[i0 + u][j0]);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float *cu = reinterpret_cast<const float *>(&cv[u]);
                        float o4[4];
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            float p = 0.f, q = 0.f;
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                p = fmaf(reinterpret_cast<const float *>(&pc[c])[u], reinterpret_cast<const float *>(&rc[c])[v], p);
                                q = fmaf(reinterpret_cast<const float *>(&pc[c + 4])[u],
                                         reinterpret_cast<const float *>(&rc[c + 4])[v], q);
                            }
                            o4[v] = (I != J || v <= u) ? cu[v] - (p + q) : cu[v];
                        }
                        *reinterpret_cast<float4 *>(&L[i0 + u][j0]) = make_float4(o4[0], o4[1], o4[2], o4[3]);
                    }
                }
            }
            bar_factor();
        }
        if (tid == 0) {
            __threadfence_block();
            *(volatile int *)&sh->prog = 1 << 20;  // done (or failed): release the inverse warps
        }
    } else {
        // ---- inverse factor (warps 8-13).  Right-looking on L X = I by block rows:
        // block row i of X accumulates T_i = sum_{j < i} L_ij X_j in place
        // (step j adds L_ij X_j once the panel of step j is final), then
        // X_i = -X_ii T_i.  So each step's share follows the factorisation's
        // step instead of piling up at the end.
        const int w = warp - 8;  // 0 .. 5
        const int u = 32 * w + lane;
        for (int j = 0; j < LB / 8; ++j) {
            const long long t0 = clock64();
            bool timed_out = false;
            while (*(volatile int *)&sh->prog < j + 1) {
                if (clock64() - t0 > wait_cycles) {
                    timed_out = true;
                    break;
                }
            }
            __threadfence_block();  // the factorisation's writes before its progress mark
            if (timed_out) sh->ifail = 1;
            if (bar_inverse_any(timed_out || *(volatile int *)&sh->fail != 0)) break;
            const int j0 = 8 * j;
            // X_j = -X_jj T_j over the columns c < j0, one thread per column
            if (u < j0) {  // (j0 <= 120 < 192 threads: one column each)
                float xd[8][8];  // X_jj (lower), the same for every thread
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int b = 0; b <= a; ++b) xd[a][b] = X[j0 + a][j0 + b];
                for (int c = u; c < j0; c += 192) {
                    float t8[8];
#pragma unroll
                    for (int b = 0; b < 8; ++b) t8[b] = X[j0 + b][c];
#pragma unroll
                    for (int a = 0; a < 8; ++a) {
                        float acc = 0.f;
#pragma unroll
                        for (int b = 0; b <= a; ++b) acc = fmaf(xd[a][b], t8[b], acc);
                        X[j0 + a][c] = -acc;
                    }
                }
            }
            if (j + 1 == LB / 8) break;
            bar_inverse();  // block row j is final
            // T_r += L[r][j0 .. j0 + 7] X_j for rows r >= j0 + 8, columns c <
            // j0 + 8: column chunks of 32 over the warps, and the rows split
            // between the warps a chunk leaves free
            const int ncols = j0 + 8, ncc = (ncols + 31) / 32, ng = 6 / ncc;
            if (w < ncc * ng) {
                const int c = 32 * (w % ncc) + lane, g = w / ncc;
                const int R = LB - ncols, per = (R + ng - 1) / ng;
                const int rb = ncols + g * per, re = min(rb + per, LB);
                if (c < ncols) {
                    float xj[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) xj[t] = X[j0 + t][c];
                    // four rows in flight (all loads before the stores), two
                    // partial sums per row
                    for (int r = rb; r < re; r += 4) {
                        float4 l0[4], l1[4];
                        float cur[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int rr = r + k < re ? r + k : r;
                            l0[k] = *reinterpret_cast<const float4 *>(&L[rr][j0]);
                            l1[k] = *reinterpret_cast<const float4 *>(&L[rr][j0 + 4]);
                            cur[k] = X[rr][c];
                        }
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            float p = fmaf(l0[k].x, xj[0], cur[k]), q = l1[k].x * xj[4];
                            p = fmaf(l0[k].y, xj[1], p);
                            q = fmaf(l1[k].y, xj[5], q);
                            p = fmaf(l0[k].z, xj[2], p);
                            q = fmaf(l1[k].z, xj[6], q);
                            p = fmaf(l0[k].w, xj[3], p);
                            q = fmaf(l1[k].w, xj[7], q);
                            if (r + k < re) X[r + k][c] = p + q;
                        }
                    }
                }
            }
            bar_inverse();  // the accumulators are updated before block row j + 1 is formed
        }
    }
    __syncthreads();
    const int fail = sh->fail ? sh->fail : (sh->ifail ? -1 : 0);
    if (fail) return fail;
    for (int r = tid; r < s; r += LT) ldiag[o + r] = (double)L[r][r];
    // X rows with 16-byte stores (zeros above the diagonal)
    for (int idx = tid; idx < LB * LB / 4; idx += LT) {
        const int r = idx / (LB / 4), c4 = 4 * (idx % (LB / 4));
        if (r >= s || c4 >= s) continue;
        const float4 v = *reinterpret_cast<const float4 *>(&X[r][c4]);
        float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (c4 + k > r) e[k] = 0.f;
        if (c4 + 3 < s) {
            *reinterpret_cast<float4 *>(Xo + (o + r) * ld + o + c4) = make_float4(e[0], e[1], e[2], e[3]);
        } else {
            for (int k = 0; k < 4 && c4 + k < s; ++k) Xo[(o + r) * ld + o + c4 + k] = e[k];
        }
    }
    return 0;
}

// After leaf_factor returned 0 (all LT threads): Xt = X^T of the block, staged
// in L's space with stride LB + 1 (conflict-free transposition), then rows of
// X^T with 16-byte stores.
__device__ __forceinline__ void leaf_store_xt(int64_t ld, int64_t o, int s, float *__restrict__ Xto,
                                              float *lsm) {
    float(*X)[LP] = reinterpret_cast<float(*)[LP]>(lsm + LB * LP);
    float *Lt = lsm;
    constexpr int LTS = LB + 1;
    const int tid = threadIdx.x;
    __syncthreads();  // L's space is free (ldiag has been read)
    for (int idx = tid; idx < LB * LB; idx += LT) {
        const int r = idx / LB, cc = idx % LB;
        Lt[cc * LTS + r] = (cc <= r) ? X[r][cc] : 0.f;  // Lt[c][r] = X[r][c] (lower X)
    }
    __syncthreads();
    for (int idx = tid; idx < LB * LB / 4; idx += LT) {
        const int r = idx / (LB / 4), c4 = 4 * (idx % (LB / 4));
        if (r >= s || c4 >= s) continue;
        const float *row = Lt + r * LTS + c4;
        if (c4 + 3 < s) {
            *reinterpret_cast<float4 *>(Xto + (o + r) * ld + o + c4) = make_float4(row[0], row[1], row[2], row[3]);
        } else {
            for (int k = 0; k < 4 && c4 + k < s; ++k) Xto[(o + r) * ld + o + c4 + k] = row[k];
        }
    }
}

}  // namespace leaf
}  // namespace glx
