// Coordinate-descent sweeps on the Newton LASSO of eq. Quad_MLE_l1_prior,
//   min_Delta tr(Delta G) + 1/2 tr(Delta W Delta W) + lambda ||A + Delta||_1,
// restricted to a pair list, keeping U = Delta W (Section 5.2: with W known
// the Hessian term costs O(|F| n)).  Coordinate (i, j) takes the exact 1-D
// minimiser of eq. 1d_l1, mu = -c + S_{lambda/a}(c - b/a), with
//   a = W_ij^2 + W_ii W_jj (W_ii^2 on the diagonal), c = A_ij + Delta_ij,
//   b = G_ij + (W Delta W)_ij,
// and the update U_i,: += mu W_j,:, U_j,: += mu W_i,: (one row on the diagonal).
//
// The sweep is a serial Gauss-Seidel chain.  It is run in blocks of B = 128
// consecutive coordinates without changing its result (up to rounding), all
// blocks of all sweeps inside one persistent cooperative launch:
//  1. dots: b0_t = G_t + W_{j_t,:} . U_{:,i_t} with U as it was before the block
//     ((W Delta W) is symmetric, so the j-row / i-column form is used), and the
//     exact interaction of an update of an earlier coordinate s on a later t,
//     K[s][t] = (W E_s W)_{i_t j_t} = W_{i_t i_s} W_{j_s j_t} + W_{i_t j_s} W_{i_s j_t}
//     (one term when s is diagonal);
//  2. resolution: for t = 0..B-1, b_t = b0_t + sum_{s<t} mu_s K[s][t] and mu_t
//     from the closed form; every CTA runs this chain itself;
//  3. row updates: each target row of U gets its updates in sweep order.
#include <math.h>

#include <algorithm>

#include "glasso_internal.h"

namespace glx {
namespace {

constexpr int DCH = 256;        // columns per dot task
constexpr int RT = 256;         // threads per CTA
constexpr int NE = 2 * CD_B;    // row-update entries per block

template <typename CT>
__device__ __forceinline__ CT soft(CT x, CT t) {
    CT ax = fabs(x) - t;
    return ax > (CT)0 ? copysign(ax, x) : (CT)0;
}

// ---------------------------------------------------------------------------
// Persistent form of the same blocked sweep: one cooperative launch runs all
// blocks of all sweeps.  Per block of B coordinates:
//   1. every CTA applies the previous block's row updates to U (work split
//      over (target row, column) items; a row's updates in sweep order);
//   -- grid barrier --
//   2. stale dots b0_t (one warp per coordinate) and the interaction matrix;
//   -- grid barrier --
//   3. every CTA loads b0 and K and runs the serial resolution itself: the
//      arithmetic is identical in every CTA, so all hold the same mu_t and the
//      same update list without a broadcast (CTA 0 alone writes Delta, after
//      the next barrier, when no CTA still reads it).
// The barrier is a monotonic arrival counter in global memory: the k-th
// barrier of the launch completes when the counter reaches k G (no reset, so
// the last CTA to arrive has nothing more to do).  Every wait is bounded
// (about 2 s of SM cycles) and sets an error word read by the host.
struct GridBar {
    unsigned count;
    unsigned unused;
    int err;
    int pad;
};

__device__ __forceinline__ void red_release_gpu(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// `epoch` counts the barriers this CTA has passed in the launch.  Arrival is a
// release reduction (no round trip); the wait polls with acquire loads.
__device__ bool grid_sync(GridBar *gb, unsigned nblocks, unsigned &epoch) {
    __shared__ int ok_s;
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) {
        volatile int *verr = &gb->err;
        const unsigned target = epoch * nblocks;
        red_release_gpu(&gb->count, 1u);
        int ok = 1;
        const long long t0 = clock64();
        while ((int)(ld_acquire_gpu(&gb->count) - target) < 0) {
            if (*verr || clock64() - t0 > 4000000000ll) {  // about 2 s
                ok = 0;
                atomicExch(&gb->err, 1);
                break;
            }
        }
        ok_s = ok && !*verr;
    }
    __syncthreads();
    return ok_s != 0;
}

// Bulk asynchronous copy of the interaction matrix into shared memory,
// completed on an mbarrier (bounded waits).
__device__ __forceinline__ uint32_t cd_smem(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void kcopy_issue(void *dst, const void *src, uint32_t bytes,
                                            unsigned long long *bar) {
    asm volatile("fence.proxy.async;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cd_smem(bar)),
                 "r"(bytes)
                 : "memory");
    constexpr uint32_t CH = 16384;
    for (uint32_t o = 0; o < bytes; o += CH)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                cd_smem(dst) + o),
            "l"((const unsigned char *)src + o), "r"(bytes - o < CH ? bytes - o : CH), "r"(cd_smem(bar))
            : "memory");
}
__device__ __forceinline__ bool kcopy_wait(unsigned long long *bar, uint32_t parity) {
    const uint32_t a = cd_smem(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > 400000000ll) return false;  // about 0.2 s
    }
}

// FP32 resolution of one block by one warp, in sub-blocks of SB coordinates.
// Lane l keeps b of coordinates l, l + 32, l + 64, l + 96.  For a sub-block,
// every lane takes a copy of its SB values (shuffles), so each step's
// dependent path is the closed form plus one FMA with no broadcast; then each
// lane adds the sub-block's SB terms to its own coordinates.  Every b_t
// receives its terms K[s][t] mu_s in ascending s, as in the lane-owner form
// (lanes also update coordinates already resolved; those values are unused).
__device__ __forceinline__ void resolve_f32(const float *__restrict__ Ks, const float *bsh,
                                            const float *csh, const float *ish, float lam,
                                            int nb, float *mush, int *zsh) {
    const int lane = threadIdx.x & 31;
    constexpr int NQ = CD_B / 32, SB = 8;
    float bl[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) bl[q] = bsh[lane + 32 * q];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
#pragma unroll
        for (int h = 0; h < 32 / SB; ++h) {
            const int t0 = 32 * q + SB * h;
            if (t0 >= nb) break;
            float bc[SB], mu[SB];
#pragma unroll
            for (int k = 0; k < SB; ++k) bc[k] = __shfl_sync(0xffffffffu, bl[q], SB * h + k);
#pragma unroll
            for (int k = 0; k < SB; ++k) {
                // coordinates t >= nb hold zeros and take mu = 0
                const int t = t0 + k;
                const float c = csh[t], ia = ish[t];
                const float x = c - bc[k] * ia;
                const float th = lam * ia;
                const float z = x - fminf(fmaxf(x, -th), th);  // S_th(x), exact zero inside
                const float m = (t < nb) ? z - c : 0.0f;
                if (lane == (t & 31)) {
                    mush[t] = m;
                    zsh[t] = (z == 0.0f);
                }
#pragma unroll
                for (int g = (k + 1) / 4; g < SB / 4; ++g) {
                    const float4 kv = *reinterpret_cast<const float4 *>(Ks + t * CD_B + t0 + 4 * g);
                    if (4 * g > k) bc[4 * g] = fmaf(kv.x, m, bc[4 * g]);
                    if (4 * g + 1 > k) bc[4 * g + 1] = fmaf(kv.y, m, bc[4 * g + 1]);
                    if (4 * g + 2 > k) bc[4 * g + 2] = fmaf(kv.z, m, bc[4 * g + 2]);
                    if (4 * g + 3 > k) bc[4 * g + 3] = fmaf(kv.w, m, bc[4 * g + 3]);
                }
                mu[k] = m;
            }
#pragma unroll
            for (int qq = q; qq < NQ; ++qq) {
                const float *Kr = Ks + t0 * CD_B + 32 * qq + lane;
#pragma unroll
                for (int k = 0; k < SB; ++k) bl[qq] = fmaf(Kr[k * CD_B], mu[k], bl[qq]);
            }
        }
    }
}

template <typename T, typename CT>
__global__ void __launch_bounds__(RT, 1) k_cd_persist(
    const T *__restrict__ W, T *__restrict__ U, int64_t n, double lam,
    const int32_t *__restrict__ pi, const int32_t *__restrict__ pj, int64_t np,
    const double *__restrict__ inva, const double *__restrict__ g, const double *__restrict__ aval,
    double *__restrict__ D, int nsweeps, double *__restrict__ bvec, double *__restrict__ Kt,
    CT *__restrict__ Kall, GridBar *gb) {
    extern __shared__ __align__(16) unsigned char ks_raw[];
    CT *Ks = reinterpret_cast<CT *>(ks_raw);  // Ks[s * CD_B + t]
    __shared__ CT bsh[CD_B], csh[CD_B], ish[CD_B], mush[CD_B];
    __shared__ int zsh[CD_B];
    __shared__ double meff[CD_B], dnew[CD_B];
    __shared__ int si[CD_B], sj[CD_B];
    __shared__ unsigned skey[NE];
    __shared__ int sdest[NE], ssrc[NE];
    __shared__ T smu[NE];  // row-update multipliers in the arithmetic of W and U
    __shared__ int seg_start[NE + 1], seg_dest[NE];
    __shared__ int nseg_s, wtot[RT / 32];
    __shared__ __align__(8) unsigned long long kbar;
    __shared__ int kok;
    unsigned epoch = 0, kuse = 0;
    constexpr uint32_t KBYTES = CD_B * CD_B * sizeof(CT);
    const unsigned G = gridDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t gthread = (int64_t)blockIdx.x * RT + tid, nthreads = (int64_t)G * RT;
    const int64_t gwarp = (int64_t)blockIdx.x * (RT / 32) + warp, nwarps = (int64_t)G * (RT / 32);
    const int64_t nbatch = (np + CD_B - 1) / CD_B;
    const int64_t total = nbatch * nsweeps;
    int64_t prev_b0 = -1;
    int prev_nb = 0;
    if (tid == 0) {
        nseg_s = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cd_smem(&kbar)), "r"(1u));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // 0. with Kall: the interaction matrices of all blocks (they depend on W
    //    and the pair list only, so every sweep reuses them); zero outside s < t < nb
    if (Kall) {
        const int64_t ktot = nbatch * (int64_t)CD_B * CD_B;
        for (int64_t q = gthread; q < ktot; q += nthreads) {
            const int64_t bb = q / (CD_B * CD_B);
            const int r = (int)(q - bb * CD_B * CD_B), s = r / CD_B, t = r - s * CD_B;
            const int64_t kb0 = bb * CD_B;
            double v = 0.0;
            if (s < t && kb0 + t < np) {
                const int64_t is = pi[kb0 + s], js = pj[kb0 + s], it2 = pi[kb0 + t], jt = pj[kb0 + t];
                v = (double)W[it2 * n + is] * (double)W[js * n + jt];
                if (is != js) v = fma((double)W[it2 * n + js], (double)W[is * n + jt], v);
            }
            Kall[q] = (CT)v;
        }
    }
    __syncthreads();
    for (int64_t it = 0; it <= total; ++it) {
        // 1. row updates of the previous block
        const int nseg = nseg_s;
        if (nseg > 0) {
            // items: (segment, group of 4 columns spaced by ncg), 32-bit index math
            const int ncg = (int)((n + 3) / 4);
            const int items = nseg * ncg;
            for (int q = (int)gthread; q < items; q += (int)nthreads) {
                const int k = q / ncg, c0 = q - k * ncg;
                T *ur = U + (int64_t)seg_dest[k] * n;
                T u[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int64_t col = c0 + (int64_t)r * ncg;
                    u[r] = col < n ? ur[col] : (T)0;
                }
                for (int e = seg_start[k]; e < seg_start[k + 1]; ++e) {
                    const T m = smu[e];
                    const T *wr = W + (int64_t)ssrc[e] * n;
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int64_t col = c0 + (int64_t)r * ncg;
                        if (col < n) u[r] = fma(m, wr[col], u[r]);
                    }
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int64_t col = c0 + (int64_t)r * ncg;
                    if (col < n) ur[col] = u[r];
                }
            }
        }
        if (it == total) break;
        if (!grid_sync(gb, G, epoch)) return;
        if (blockIdx.x == 0 && prev_b0 >= 0)
            for (int t = tid; t < prev_nb; t += RT) D[prev_b0 + t] = dnew[t];
        const int64_t b0 = (it % nbatch) * CD_B;
        const int nb = (int)lmin(CD_B, np - b0);
        if (Kall && tid == 0) kcopy_issue(Ks, Kall + (it % nbatch) * CD_B * CD_B, KBYTES, &kbar);
        // 2. stale dots as (coordinate, chunk of DCH columns) warp tasks, partial
        //    sums per chunk (summed in a fixed order in step 3); interactions
        const int nch = (int)((n + DCH - 1) / DCH);
        for (int64_t task = gwarp; task < (int64_t)nb * nch; task += nwarps) {
            const int t = (int)(task / nch), c = (int)(task - (int64_t)t * nch);
            const int64_t it_ = pi[b0 + t], jt = pj[b0 + t];
            const T *wr = W + jt * n;
            const T *uc = U + it_;
            const int64_t k0 = (int64_t)c * DCH, k1 = lmin(n, k0 + DCH);
            T acc = 0;
#pragma unroll 8
            for (int64_t k = k0 + lane; k < k1; k += 32) acc = fma(wr[k], uc[k * n], acc);
            // warp sum in the arithmetic of W and U (FP64 operations and
            // conversions run at a small fraction of the FP32 rate on this
            // GPU); the chunk partials are summed in FP64
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) bvec[(int64_t)c * CD_B + t] = (double)acc;
        }
        CT *Ktc = reinterpret_cast<CT *>(Kt);
        for (int q = (int)gthread; !Kall && q < nb * nb; q += (int)nthreads) {
            const int s = q / nb, t = q - s * nb;
            if (s < t) {
                const int64_t is = pi[b0 + s], js = pj[b0 + s], it2 = pi[b0 + t], jt = pj[b0 + t];
                double v = (double)W[it2 * n + is] * (double)W[js * n + jt];
                if (is != js) v = fma((double)W[it2 * n + js], (double)W[is * n + jt], v);
                Ktc[s * CD_B + t] = (CT)v;
            }
        }
        if (!grid_sync(gb, G, epoch)) {
            if (Kall && tid == 0) kcopy_wait(&kbar, kuse & 1u);  // the prefetch in flight
            return;
        }
        if (!Kall && tid == 0) kcopy_issue(Ks, Ktc, KBYTES, &kbar);
        // 3. resolution, identical in every CTA
        if (tid < nb) {
            // independent loads of the chunk partials, summed in chunk order
            double b = g[b0 + tid];
            int c = 0;
            for (; c + 8 <= nch; c += 8) {
                double v[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) v[r] = bvec[(int64_t)(c + r) * CD_B + tid];
#pragma unroll
                for (int r = 0; r < 8; ++r) b += v[r];
            }
            for (; c < nch; ++c) b += bvec[(int64_t)c * CD_B + tid];
            bsh[tid] = (CT)b;
            csh[tid] = (CT)(aval[b0 + tid] + D[b0 + tid]);
            ish[tid] = (CT)inva[b0 + tid];
            si[tid] = pi[b0 + tid];
            sj[tid] = pj[b0 + tid];
        } else if (tid < CD_B) {
            bsh[tid] = csh[tid] = ish[tid] = (CT)0;
            si[tid] = sj[tid] = 0;
        }
        if (tid == 0) {
            const bool got = kcopy_wait(&kbar, kuse & 1u);
            if (!got) {
                atomicExch(&gb->err, 1);
                kcopy_wait(&kbar, kuse & 1u);  // let the copy land before leaving
            }
            kok = got;
        }
        ++kuse;
        __syncthreads();
        if (!kok) return;
        if (tid < 32) {
            if constexpr (sizeof(CT) == 4) {
                resolve_f32(reinterpret_cast<const float *>(Ks), reinterpret_cast<const float *>(bsh),
                            reinterpret_cast<const float *>(csh), reinterpret_cast<const float *>(ish),
                            (float)lam, nb, reinterpret_cast<float *>(mush), zsh);
            } else {
                // lane l holds b, c, 1/a of coordinates l, l+32, l+64, l+96 in registers;
                // the owner of coordinate t computes mu_t and broadcasts it by shuffle
                CT br[CD_B / 32], cr[CD_B / 32], ir[CD_B / 32];
#pragma unroll
                for (int q = 0; q < CD_B / 32; ++q) {
                    br[q] = bsh[lane + 32 * q];
                    cr[q] = csh[lane + 32 * q];
                    ir[q] = ish[lane + 32 * q];
                }
                const CT lamc = (CT)lam;
#pragma unroll
                for (int q = 0; q < CD_B / 32; ++q) {
#pragma unroll 4
                    for (int tt = 0; tt < 32; ++tt) {
                        const int t = 32 * q + tt;
                        if (t >= nb) break;
                        CT mu = 0;
                        int zf = 0;
                        if (lane == tt) {
                            const CT z = soft(cr[q] - br[q] * ir[q], lamc * ir[q]);
                            mu = z - cr[q];
                            zf = (z == (CT)0);
                            mush[t] = mu;
                            zsh[t] = zf;
                        }
                        mu = __shfl_sync(0xffffffffu, mu, tt);
                        if (mu != (CT)0) {
                            const CT *kr = Ks + t * CD_B;
#pragma unroll
                            for (int qq = q; qq < CD_B / 32; ++qq) {
                                const int s2 = lane + 32 * qq;
                                if (s2 > t) br[qq] = fma(kr[s2], mu, br[qq]);
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (tid < nb) {
            const double d0 = D[b0 + tid];
            double m = 0.0, dn = d0;
            if (mush[tid] != (CT)0) {
                if (zsh[tid]) {
                    dn = -aval[b0 + tid];
                    m = dn - d0;
                } else {
                    m = (double)mush[tid];
                    dn = d0 + m;
                }
            }
            meff[tid] = m;
            dnew[tid] = dn;
        }
        __syncthreads();
        // row updates: entry e = 2t + k (k = 0: row i_t gets mu W_{j_t}; k = 1: row
        // j_t gets mu W_{i_t}); sort the packed keys (target row, e) so that the
        // updates of a row are contiguous and in sweep order
        unsigned key = 0xFFFFFFFFu;
        {
            const int e = tid, t = e >> 1, k = e & 1;  // RT == NE
            if (t < nb && meff[t] != 0.0) {
                if (k == 0) key = ((unsigned)si[t] << 9) | (unsigned)e;
                else if (si[t] != sj[t]) key = ((unsigned)sj[t] << 9) | (unsigned)e;
            }
        }
        // bitonic sort, one key per thread: partners inside a warp by shuffle,
        // across warps through shared memory
        for (int size = 2; size <= NE; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                unsigned other;
                if (stride >= 32) {
                    skey[tid] = key;
                    __syncthreads();
                    other = skey[tid ^ stride];
                    __syncthreads();
                } else {
                    other = __shfl_xor_sync(0xffffffffu, key, stride);
                }
                const bool up = (tid & size) == 0, lower = (tid & stride) == 0;
                key = (lower == up) ? min(key, other) : max(key, other);
            }
        }
        int V = 0;
        {
            const unsigned kk = key;
            const int valid = kk != 0xFFFFFFFFu;
            if (valid) {
                const int e = (int)(kk & 511u), t = e >> 1;
                sdest[tid] = (int)(kk >> 9);
                ssrc[tid] = (e & 1) ? si[t] : sj[t];
                smu[tid] = (T)meff[t];
            }
            int v = valid;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) wtot[warp] = v;
            __syncthreads();
            for (int w2 = 0; w2 < RT / 32; ++w2) V += wtot[w2];
            __syncthreads();
        }
        const int r = tid;  // RT == NE
        const int start = (r < V) && (r == 0 || sdest[r] != sdest[r - 1]);
        int x = start;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wtot[warp] = x;
        __syncthreads();
        int before = 0, nsg = 0;
        for (int w2 = 0; w2 < RT / 32; ++w2) {
            if (w2 < warp) before += wtot[w2];
            nsg += wtot[w2];
        }
        const int idx = before + x - start;
        if (start) {
            seg_start[idx] = r;
            seg_dest[idx] = sdest[r];
        }
        if (tid == 0) {
            nseg_s = nsg;
            seg_start[nsg] = V;
        }
        __syncthreads();
        prev_b0 = b0;
        prev_nb = nb;
    }
    if (blockIdx.x == 0 && prev_b0 >= 0)
        for (int t = tid; t < prev_nb; t += RT) D[prev_b0 + t] = dnew[t];
}

bool g_attr_done[4] = {false, false, false, false};

}  // namespace

template <typename T, typename CT>
static cudaError_t cd_sweeps_t(const T *W, int64_t n, double lam, const int32_t *pi,
                               const int32_t *pj, int64_t np, const double *inva, const double *g,
                               const double *aval, int nsweeps, double *D, T *U, Work &w,
                               cudaStream_t st) {
    static_assert(RT == NE, "one entry per thread in resolve");
    if (n > (1 << 22)) return cudaErrorInvalidValue;  // packed sort keys hold the row in 23 bits
    const size_t kbytes = (size_t)CD_B * CD_B * sizeof(CT);
    const int which = (sizeof(T) == 8 ? 2 : 0) + (sizeof(CT) == 8 ? 1 : 0);
    static int nsm = 0, occ[4] = {0, 0, 0, 0};
    if (!g_attr_done[which]) {
        cudaError_t e = cudaFuncSetAttribute(k_cd_persist<T, CT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kbytes);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[which], k_cd_persist<T, CT>, RT, kbytes);
        if (e != cudaSuccess) return e;
        if (occ[which] < 1) return cudaErrorInvalidConfiguration;
        g_attr_done[which] = true;
    }
    if (np <= 0 || nsweeps <= 0) return cudaSuccess;
    // enough CTAs for the row-update and dot phases, no more than co-resident
    int G = (int)lmax(4, lmin((int64_t)nsm * occ[which], (n + 7) / 8));
    // partial dots: ceil(n / DCH) x CD_B doubles, then the interaction matrix
    if ((n + DCH - 1) / DCH > CD_MAX_CHUNKS) return cudaErrorInvalidValue;
    double *bvec = w.cd_part;
    double *Kt = w.cd_part + (size_t)CD_MAX_CHUNKS * CD_B;
    static_assert(sizeof(GridBar) == 4 * sizeof(int), "barrier words");
    GridBar *gb = reinterpret_cast<GridBar *>(&w.sc->bar_count);
    cudaError_t e = cudaMemsetAsync(gb, 0, sizeof(GridBar), st);
    if (e != cudaSuccess) return e;
    // interaction matrices of all blocks, computed once per launch, while they
    // fit in n^2 doubles (else each block computes its own)
    const size_t kneed = (size_t)((np + CD_B - 1) / CD_B) * kbytes;
    CT *Kall = nullptr;
    if (kneed <= (size_t)n * (size_t)n * sizeof(double)) {
        if (w.cap_cd_k < kneed) {
            const size_t want = std::min((size_t)n * (size_t)n * sizeof(double),
                                         std::max(kneed, 2 * w.cap_cd_k));
            if (w.cd_k) {
                e = cudaFreeAsync(w.cd_k, st);
                w.cd_k = nullptr;
                w.cap_cd_k = 0;
                if (e != cudaSuccess) return e;
            }
            e = cudaMallocAsync((void **)&w.cd_k, want, st);
            if (e != cudaSuccess) return e;
            w.cap_cd_k = want;
        }
        Kall = reinterpret_cast<CT *>(w.cd_k);
    }
    void *args[] = {(void *)&W, (void *)&U, (void *)&n, (void *)&lam, (void *)&pi, (void *)&pj,
                    (void *)&np, (void *)&inva, (void *)&g, (void *)&aval, (void *)&D,
                    (void *)&nsweeps, (void *)&bvec, (void *)&Kt, (void *)&Kall, (void *)&gb};
    e = cudaLaunchCooperativeKernel((const void *)k_cd_persist<T, CT>, dim3(G), dim3(RT), args,
                                    kbytes, st);
    counted(1);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t cd_sweeps(const double *W, int64_t n, double lam, const int32_t *pi,
                      const int32_t *pj, int64_t np, const double *inva, const double *g,
                      const double *aval, int nsweeps, double *D, double *U, Work &w,
                      cudaStream_t st) {
    return cd_sweeps_t<double, double>(W, n, lam, pi, pj, np, inva, g, aval, nsweeps, D, U, w, st);
}

cudaError_t cd_sweeps32(const float *W, int64_t n, double lam, const int32_t *pi,
                        const int32_t *pj, int64_t np, const double *inva, const double *g,
                        const double *aval, int nsweeps, double *D, float *U, Work &w,
                        bool chain64, cudaStream_t st) {
    if (chain64)
        return cd_sweeps_t<float, double>(W, n, lam, pi, pj, np, inva, g, aval, nsweeps, D, U, w, st);
    return cd_sweeps_t<float, float>(W, n, lam, pi, pj, np, inva, g, aval, nsweeps, D, U, w, st);
}

}  // namespace glx
