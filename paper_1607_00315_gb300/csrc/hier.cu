// Multilevel hierarchy of Section 3.2 / Section 7: nested coarse sets
//   C_1 > C_2 > ... > C_L = supp(A^(k)),
//   |C_1| = max(ceil(|F_k|/2), |supp|), |C_{l+1}| = max(ceil(|C_l|/2), |supp|),
// each C_l = supp + the non-support pairs of F_k with the largest |G|
// (ties: earlier pair in the list first).  Output: per pair the coarsest
// level that contains it (a level tag).
//
// The ranking only matters at the L thresholds |C_l| - |supp|, so instead of
// sorting, one CTA finds each threshold key by an 8-bit MSD radix select on
// the IEEE bit pattern of |G| (non-negative doubles order like their bits),
// then assigns tags in one ordered pass; equal keys at a threshold are split
// by their list position with a block-wide prefix count.
#include "glasso_internal.h"

namespace glx {
namespace {

constexpr int HT = 1024;
constexpr int MAXL = 62;

__device__ __forceinline__ unsigned long long keyof(const double *absg, int64_t p) {
    return (unsigned long long)__double_as_longlong(absg[p]);
}

__device__ long long block_sum_ll(long long v, long long *scratch32) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) scratch32[threadIdx.x >> 5] = v;
    __syncthreads();
    long long s = 0;
    for (int w = 0; w < HT / 32; ++w) s += scratch32[w];
    __syncthreads();
    return s;
}

__device__ long long block_exscan_ll(long long v, long long *total, long long *scratch32) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) scratch32[wid] = x;
    __syncthreads();
    long long before = 0, tot = 0;
    for (int w = 0; w < HT / 32; ++w) {
        if (w < wid) before += scratch32[w];
        tot += scratch32[w];
    }
    __syncthreads();
    *total = tot;
    return before + x - v;
}

__global__ void __launch_bounds__(HT) k_hierarchy(const double *__restrict__ absg,
                                                  const uint8_t *__restrict__ insupp, int64_t nf,
                                                  uint8_t *__restrict__ tag, DevScalars *sc) {
    __shared__ long long sizes[MAXL + 2];
    __shared__ unsigned long long vsel[MAXL + 2];
    __shared__ long long need[MAXL + 2], eqc[MAXL + 2], running[MAXL + 2];
    __shared__ unsigned int hist[256];
    __shared__ long long scratch[32];
    __shared__ int Ls;
    __shared__ unsigned long long sh_prefix;
    __shared__ long long sh_rem;
    const int tid = threadIdx.x;

    long long c = 0;
    for (int64_t p = tid; p < nf; p += HT) c += insupp[p] ? 1 : 0;
    const long long ns = block_sum_ll(c, scratch);
    if (tid == 0) {
        long long s = (nf + 1) / 2;
        if (s < ns) s = ns;
        sizes[1] = s;
        int L = 1;
        while (sizes[L] > ns && L < MAXL) {
            long long nx = (sizes[L] + 1) / 2;
            if (nx < ns) nx = ns;
            sizes[++L] = nx;
        }
        Ls = L;
    }
    __syncthreads();
    const int L = Ls;

    for (int l = 1; l <= L; ++l) {
        const long long t = sizes[l] - ns;  // non-support pairs in C_l
        if (t <= 0) {
            if (tid == 0) { need[l] = 0; eqc[l] = 0; vsel[l] = 0; }
            __syncthreads();
            continue;
        }
        unsigned long long prefix = 0, pmask = 0;
        long long rem = t;
        for (int shift = 56; shift >= 0; shift -= 8) {
            for (int d = tid; d < 256; d += HT) hist[d] = 0;
            __syncthreads();
            for (int64_t p = tid; p < nf; p += HT) {
                if (insupp[p]) continue;
                const unsigned long long k = keyof(absg, p);
                if ((k & pmask) == prefix) atomicAdd(&hist[(k >> shift) & 255ull], 1u);
            }
            __syncthreads();
            if (tid == 0) {
                long long cum = 0;
                int sel = 0;
                for (int d = 255; d >= 0; --d) {
                    if (cum + (long long)hist[d] >= rem) { sel = d; break; }
                    cum += hist[d];
                }
                sh_rem = rem - cum;
                sh_prefix = prefix | ((unsigned long long)sel << shift);
            }
            __syncthreads();
            prefix = sh_prefix;
            rem = sh_rem;
            pmask |= 0xFFull << shift;
            __syncthreads();
        }
        long long gt = 0, eq = 0;
        for (int64_t p = tid; p < nf; p += HT) {
            if (insupp[p]) continue;
            const unsigned long long k = keyof(absg, p);
            gt += k > prefix;
            eq += k == prefix;
        }
        gt = block_sum_ll(gt, scratch);
        eq = block_sum_ll(eq, scratch);
        if (tid == 0) {
            vsel[l] = prefix;
            need[l] = t - gt;
            eqc[l] = eq;
            running[l] = 0;
        }
        __syncthreads();
    }

    for (int64_t base = 0; base < nf; base += HT) {
        const int64_t p = base + tid;
        const bool valid = p < nf;
        const bool s = valid && insupp[p];
        const unsigned long long k = valid ? keyof(absg, p) : 0ull;
        int tg = s ? L : 0;
        for (int l = 1; l <= L; ++l) {
            if (need[l] <= 0) continue;  // uniform: no non-support pair at this level
            const bool isEq = valid && !s && k == vsel[l];
            bool in;
            if (eqc[l] > need[l]) {  // uniform: split the ties by list position
                long long tot;
                const long long r = block_exscan_ll(isEq ? 1 : 0, &tot, scratch) + running[l];
                in = (k > vsel[l]) || (isEq && r < need[l]);
                __syncthreads();
                if (tid == 0) running[l] += tot;
                __syncthreads();
            } else {
                in = (k > vsel[l]) || isEq;
            }
            if (valid && !s && in) tg = l;
        }
        if (valid) tag[p] = (uint8_t)tg;
    }
    if (tid == 0) {
        sc->levels = L;
        sc->nsupp = ns;
    }
}

}  // namespace

cudaError_t hierarchy(const double *absg, const uint8_t *insupp, int64_t nf, uint8_t *tag,
                      DevScalars *sc, cudaStream_t st) {
    if (nf < 0 || nf > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_hierarchy<<<1, HT, 0, st>>>(absg, insupp, nf, tag, sc);
    counted(1);
    return cudaGetLastError();
}

}  // namespace glx
