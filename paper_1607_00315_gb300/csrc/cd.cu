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
//     from the closed form (the FP32 chain carries x_t = c_t - b_t / a_t
//     instead of b_t); every CTA runs this chain itself;
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

// Limit of every grid-barrier wait in SM cycles, and a number of arrivals the
// barrier waits for beyond the grid (0 in normal operation; a test sets 1, so
// that the wait runs to its limit and the error path is taken).
struct WaitCfg {
    long long cycles;
    unsigned extra;
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
__device__ bool grid_sync(GridBar *gb, unsigned nblocks, unsigned &epoch, const WaitCfg &wc) {
    __shared__ int ok_s;
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) {
        volatile int *verr = &gb->err;
        const unsigned target = epoch * nblocks + wc.extra;
        red_release_gpu(&gb->count, 1u);
        int ok = 1;
        const long long t0 = clock64();
        unsigned spins = 0;
        // one acquire load per poll; the error word (a CTA that gave up) is
        // read every 32 polls
        while ((int)(ld_acquire_gpu(&gb->count) - target) < 0) {
            if ((++spins & 31u) == 0 && (*verr || clock64() - t0 > wc.cycles)) {
                ok = 0;
                atomicExch(&gb->err, 1);
                break;
            }
        }
        // (an error word set by a CTA that still arrived is left to the host,
        // which reads it after the launch: no extra round trip here)
        ok_s = ok;
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

// FP32 resolution of one block by one warp, in sub-blocks of SB coordinates,
// in the argument x_t = c_t - b_t / a_t of the closed form of eq. 1d_l1,
// mu_t = S_{lambda/a_t}(x_t) - c_t.  An update mu_s of an earlier coordinate
// changes x_t by -(K[s][t] / a_t) mu_s, so Ks holds K[s][t] / a_t (s < t, zero
// elsewhere) and no scaling sits on the dependent path.
// xsh[t] = c_t - b_t / a_t, csh[t] = c_t, thsh[t] = lam / a_t (zero for t >= nb).
// Lane l keeps x of coordinates l, l + 32, l + 64, l + 96.  For a sub-block,
// every lane takes a copy of its SB values (shuffles), so each step's
// dependent path is the clamp, two subtractions and one FMA with no
// broadcast; then each lane adds the sub-block's SB terms to its own
// coordinates.  Every x_t receives its terms in ascending s, as in the
// lane-owner form (lanes also update coordinates already resolved; those
// values are unused).  The owner lane of t keeps mu_t and the zero flag in
// registers and stores them once at the end.
__device__ __forceinline__ void resolve_f32(const float *__restrict__ Ks, const float *__restrict__ xsh,
                                            const float *__restrict__ csh,
                                            const float *__restrict__ thsh, int nb,
                                            float *__restrict__ mush, int *__restrict__ zsh) {
    const int lane = threadIdx.x & 31;
    constexpr int NQ = CD_B / 32, SB = 8;
    float xl[NQ], mown[NQ];
    int zown[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        xl[q] = xsh[lane + 32 * q];
        mown[q] = 0.f;
        zown[q] = 0;
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
#pragma unroll
        for (int h = 0; h < 32 / SB; ++h) {
            const int t0 = 32 * q + SB * h;
            if (t0 >= nb) break;
            float xc[SB], cc[SB], th[SB], mu[SB];
#pragma unroll
            for (int k = 0; k < SB; ++k) xc[k] = __shfl_sync(0xffffffffu, xl[q], SB * h + k);
#pragma unroll
            for (int k = 0; k < SB; k += 4) {
                const float4 cv = *reinterpret_cast<const float4 *>(csh + t0 + k);
                const float4 tv = *reinterpret_cast<const float4 *>(thsh + t0 + k);
                cc[k] = cv.x, cc[k + 1] = cv.y, cc[k + 2] = cv.z, cc[k + 3] = cv.w;
                th[k] = tv.x, th[k + 1] = tv.y, th[k + 2] = tv.z, th[k + 3] = tv.w;
            }
#pragma unroll
            for (int k = 0; k < SB; ++k) {
                // coordinates t >= nb hold zeros and take mu = 0
                const int t = t0 + k;
                const float z = xc[k] - fminf(fmaxf(xc[k], -th[k]), th[k]);  // exact zero inside
                const float m = (t < nb) ? z - cc[k] : 0.0f;
                if (lane == SB * h + k) {
                    mown[q] = m;
                    zown[q] = (z == 0.0f);
                }
#pragma unroll
                for (int g = (k + 1) / 4; g < SB / 4; ++g) {
                    const float4 kv = *reinterpret_cast<const float4 *>(Ks + t * CD_B + t0 + 4 * g);
                    if (4 * g > k) xc[4 * g] = fmaf(-kv.x, m, xc[4 * g]);
                    if (4 * g + 1 > k) xc[4 * g + 1] = fmaf(-kv.y, m, xc[4 * g + 1]);
                    if (4 * g + 2 > k) xc[4 * g + 2] = fmaf(-kv.z, m, xc[4 * g + 2]);
                    if (4 * g + 3 > k) xc[4 * g + 3] = fmaf(-kv.w, m, xc[4 * g + 3]);
                }
                mu[k] = m;
            }
#pragma unroll
            for (int qq = q; qq < NQ; ++qq) {
                const float *Kr = Ks + t0 * CD_B + 32 * qq + lane;
#pragma unroll
                for (int k = 0; k < SB; ++k) xl[qq] = fmaf(-Kr[k * CD_B], mu[k], xl[qq]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        mush[lane + 32 * q] = mown[q];
        zsh[lane + 32 * q] = zown[q];
    }
}

template <typename T, typename CT>
__global__ void __launch_bounds__(RT, 1) k_cd_persist(
    const T *__restrict__ W, T *__restrict__ U, int64_t n, double lam,
    const int32_t *__restrict__ pi, const int32_t *__restrict__ pj, int64_t np,
    const double *__restrict__ inva, const double *__restrict__ g, const double *__restrict__ aval,
    double *__restrict__ D, int nsweeps, double *__restrict__ bvec, double *__restrict__ Kt,
    CT *__restrict__ Kall, GridBar *gb, WaitCfg wc) {
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
            if constexpr (sizeof(CT) == 4) {  // the FP32 chain works in x (K[s][t] / a_t)
                if (s < t && kb0 + t < np) v *= inva[kb0 + t];
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
        if (!grid_sync(gb, G, epoch, wc)) return;
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
                if constexpr (sizeof(CT) == 4) v *= inva[b0 + t];
                Ktc[s * CD_B + t] = (CT)v;
            }
        }
        if (!grid_sync(gb, G, epoch, wc)) {
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
            const double cv = aval[b0 + tid] + D[b0 + tid], ia = inva[b0 + tid];
            if constexpr (sizeof(CT) == 4) {  // x, c and the threshold of the FP32 chain
                bsh[tid] = (CT)(cv - b * ia);
                csh[tid] = (CT)cv;
                ish[tid] = (CT)(lam * ia);
            } else {
                bsh[tid] = (CT)b;
                csh[tid] = (CT)cv;
                ish[tid] = (CT)ia;
            }
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
                            nb, reinterpret_cast<float *>(mush), zsh);
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

// ---------------------------------------------------------------------------
// FP32 sweep with the serial chain on one CTA and the row updates off its
// path.  CTA 0 (the chain CTA) holds the interaction matrices and resolves
// the chain; CTAs 1..G-1 (work CTAs) take the stale dots and apply the row
// updates.  Two copies of U alternate: in pass p, copy p mod 2 holds U after
// blocks < p - 1 and is only read, copy (p + 1) mod 2 holds U after blocks
// < p - 2 and is only written.  Pass p:
//   chain CTA: x of block p from its stale dots (taken in pass p - 1 against
//     U after blocks < p - 2) minus the exact terms of blocks p - 2 and p - 1,
//     (K2_{p-2})^T mu_{p-2} + (K1_{p-1})^T mu_{p-1}, where
//     Kd_q[s][t] = K(s in block q -> t in block q + d) / a_t (all s and t;
//     the block sequence wraps around the sweep); warp 0 resolves the chain
//     of block p while warps 1-8 take the term of block p - 1 on block p + 1;
//     FP64 increments with exact zeros; block p's row-update multipliers go
//     to global memory; the term of block p on block p + 1;
//   work CTAs: stale dots of block p + 1 against copy p mod 2; the row
//     updates of blocks p - 2 and p - 1 applied to copy (p + 1) mod 2, which
//     then holds U after blocks <= p - 1;
//   grid barrier.
// A last pass without a chain applies the final two blocks.  Which rows an
// update touches depends only on the pair list, so the per-launch setup
// computes, besides the intra and cross matrices, for every pair of
// consecutive blocks the list of their row updates sorted by target row
// (the earlier block first within a row) and its segments; a pass only
// looks up the multipliers (an update with multiplier 0 leaves U as it is).
constexpr int LW = 8;              // worker warps (warps 1..LW)
constexpr int LT = 32 * (LW + 1);  // warp 0 of the chain CTA runs the chain
constexpr int NWK = 32 * LW;       // worker threads
constexpr int NE2 = 2 * NE;        // row updates of two blocks
static_assert(NWK == NE && NWK == 2 * CD_B, "one entry per worker thread; cross-term halves");
// merged list of two blocks in global memory: V, nseg, src[NE2], ref[NE2],
// seg_start[NE2 + 1], seg_dest[NE2] (ref = slot * NE + entry; slot 0 = the
// earlier block); padded to a multiple of 4 words
constexpr int LST = (2 + 4 * NE2 + 1 + 3) / 4 * 4;

__device__ __forceinline__ void wsync() { asm volatile("bar.sync 1, %0;" ::"n"(NWK) : "memory"); }

__global__ void __launch_bounds__(LT, 1) k_cd_lag2(
    const float *__restrict__ W, float *__restrict__ Ubuf0, float *__restrict__ Ubuf1, int64_t n,
    double lam, const int32_t *__restrict__ pi, const int32_t *__restrict__ pj, int64_t np,
    const double *__restrict__ inva, const double *__restrict__ g, const double *__restrict__ aval,
    double *__restrict__ D, int nsweeps, double *__restrict__ bvec, float *__restrict__ Kall,
    int *__restrict__ lists, float *__restrict__ gmu, GridBar *gb, WaitCfg wc) {
    extern __shared__ __align__(16) unsigned char ks_raw[];
    // intra matrices K[s][t] / a_t (s < t) of this pass and the next (by pass
    // parity), and the block p -> p + 1 matrix; the p - 1 -> p + 1 term is
    // read from global memory by the otherwise idle worker warps
    float *KIb = reinterpret_cast<float *>(ks_raw);
    float *K1 = KIb + 2 * CD_B * CD_B;
    // chain CTA
    __shared__ __align__(16) float xsh[CD_B], csh[CD_B], thsh[CD_B];
    __shared__ float mush[CD_B], mprev[CD_B], xn[CD_B], xc2[2][CD_B], x1[2][CD_B];
    __shared__ int zsh[CD_B];
    __shared__ double meff[CD_B], dold[CD_B], aold[CD_B];
    // list setup and work CTAs
    __shared__ unsigned sx[NE];
    __shared__ int ldest[2][NE], lsrc[2][NE], lref[2][NE], lcount[2];
    __shared__ int mdest[NE2], msrc[NE2], mref[NE2];
    __shared__ float mutab[NE2];
    __shared__ int seg_start[NE2 + 1], seg_dest[NE2];
    __shared__ int nseg_s, nv_s, wtot[LW], wv[LW];
    __shared__ __align__(8) unsigned long long kbarI[2], kbar1;
    constexpr uint32_t KB = CD_B * CD_B * sizeof(float);
    const unsigned G = gridDim.x;
    const bool cc = blockIdx.x == 0;
    const int GW = (int)G - 1, wb = (int)blockIdx.x - 1;  // work CTAs
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, wtid = tid - 32;
    const int64_t nbatch = (np + CD_B - 1) / CD_B;
    const int64_t total = nbatch * nsweeps;
    const int nch = (int)((n + DCH - 1) / DCH);
    const int64_t KS = (int64_t)CD_B * CD_B;
    const float *KallI = Kall, *Kall1 = Kall + nbatch * KS, *Kall2 = Kall + 2 * nbatch * KS;
    // mbarrier phases, advanced by every thread of the chain CTA in step (the
    // waiting and the issuing threads differ); outstanding copies per issuer
    unsigned epoch = 0, phI0 = 0, phI1 = 0, ph1 = 0;
    int pendI0 = 0, pendI1 = 0, pend1 = 0;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cd_smem(&kbarI[0])), "r"(1u));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cd_smem(&kbarI[1])), "r"(1u));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cd_smem(&kbar1)), "r"(1u));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int t = tid; t < CD_B; t += LT) {
        mprev[t] = 0.f;
        xn[t] = 0.f;
    }
    auto drain = [&]() {  // let issued copies land before the CTA leaves
        if (pendI0) kcopy_wait(&kbarI[0], phI0 & 1u);
        if (pendI1) kcopy_wait(&kbarI[1], phI1 & 1u);
        if (pend1) kcopy_wait(&kbar1, ph1 & 1u);
    };
    auto kwait = [&](unsigned long long *bar, unsigned ph) {
        if (!kcopy_wait(bar, ph & 1u)) {
            atomicExch(&gb->err, 1);
            kcopy_wait(bar, ph & 1u);
        }
    };
    // 0a. interaction matrices of all blocks: intra, +1 and +2 (scaled by 1/a
    //     of the target), four entries per thread in flight
    {
        const int64_t per = nbatch * KS, tot = 3 * per;
        const int64_t gthread = (int64_t)blockIdx.x * LT + tid, nthreads = (int64_t)G * LT;
        for (int64_t q0 = gthread; q0 < tot; q0 += 4 * nthreads) {
            int64_t is[4], js[4], it2[4], jt[4], kt[4];
            bool ok[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t q = q0 + u * nthreads;
                ok[u] = false;
                if (q < tot) {
                    const int kind = (int)(q / per);
                    const int64_t qq = q - kind * per;
                    const int64_t bb = qq / KS;
                    const int r = (int)(qq - bb * KS), s = r / CD_B, t = r - s * CD_B;
                    const int64_t ks0 = bb * CD_B, kt0 = ((bb + kind) % nbatch) * CD_B;
                    ok[u] = (kind > 0 || s < t) && ks0 + s < np && kt0 + t < np;
                    kt[u] = kt0 + t;
                    if (ok[u]) {
                        is[u] = pi[ks0 + s];
                        js[u] = pj[ks0 + s];
                        it2[u] = pi[kt0 + t];
                        jt[u] = pj[kt0 + t];
                    }
                }
            }
            float w1[4], w2[4], w3[4], w4[4];
            double ia[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (ok[u]) {
                    w1[u] = W[it2[u] * n + is[u]];
                    w2[u] = W[js[u] * n + jt[u]];
                    w3[u] = W[it2[u] * n + js[u]];
                    w4[u] = W[is[u] * n + jt[u]];
                    ia[u] = inva[kt[u]];
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t q = q0 + u * nthreads;
                if (q < tot) {
                    double v = 0.0;
                    if (ok[u]) {
                        v = (double)w1[u] * (double)w2[u];
                        if (is[u] != js[u]) v = fma((double)w3[u], (double)w4[u], v);
                        v *= ia[u];
                    }
                    Kall[q] = (float)v;
                }
            }
        }
    }
    // 0b. merged row-update lists: list L < nbatch holds blocks (L - 1) mod
    //     nbatch (slot 0) and L (slot 1); list nbatch holds block 0 alone
    //     (slot 1).  Entry e = 2t + k of a block updates row i_t from row j_t
    //     (k = 0) or row j_t from row i_t (k = 1, off-diagonal pairs only).
    if (warp > 0) {
        for (int64_t L = blockIdx.x; L <= nbatch; L += G) {
#pragma unroll 1
            for (int slot = 0; slot < 2; ++slot) {
                const bool has = slot == 1 || L < nbatch;
                const int64_t q = slot == 1 ? (L < nbatch ? L : 0) : (L + nbatch - 1) % nbatch;
                const int64_t q0 = q * CD_B;
                const int nbq = (int)lmin(CD_B, np - q0);
                const int e = wtid, t = e >> 1, k = e & 1;
                unsigned key = 0xFFFFFFFFu;
                int src = 0;
                if (has && t < nbq) {
                    const int i_ = pi[q0 + t], j_ = pj[q0 + t];
                    src = k ? i_ : j_;
                    if (k == 0) key = ((unsigned)i_ << 9) | (unsigned)e;
                    else if (i_ != j_) key = ((unsigned)j_ << 9) | (unsigned)e;
                }
                lsrc[slot][e] = src;  // by entry, gathered after the sort
                for (int size = 2; size <= NE; size <<= 1) {
                    for (int stride = size >> 1; stride > 0; stride >>= 1) {
                        unsigned other;
                        if (stride >= 32) {
                            sx[wtid] = key;
                            wsync();
                            other = sx[wtid ^ stride];
                            wsync();
                        } else {
                            other = __shfl_xor_sync(0xffffffffu, key, stride);
                        }
                        const bool up = (wtid & size) == 0, lower = (wtid & stride) == 0;
                        key = (lower == up) ? min(key, other) : max(key, other);
                    }
                }
                const bool valid = key != 0xFFFFFFFFu;
                const int v = __popc(__ballot_sync(0xffffffffu, valid));
                if (lane == 0) wv[warp - 1] = v;
                int ssrc = 0, sref = 0;
                if (valid) {
                    const int ee = (int)(key & 511u);
                    ssrc = lsrc[slot][ee];
                    sref = slot * NE + ee;
                }
                wsync();
                if (valid) {
                    ldest[slot][wtid] = (int)(key >> 9);
                    lsrc[slot][wtid] = ssrc;
                    lref[slot][wtid] = sref;
                }
                if (wtid == 0) {
                    int V = 0;
                    for (int w2 = 0; w2 < LW; ++w2) V += wv[w2];
                    lcount[slot] = V;
                }
                wsync();
            }
            // merge: slot 0 before slot 1 within a row (binary search placement)
            const int VP = lcount[0], VC = lcount[1];
            if (wtid < VP) {
                const int d = ldest[0][wtid];
                int lo = 0, hi = VC;  // slot-1 entries with dest < d
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (ldest[1][mid] < d) lo = mid + 1;
                    else hi = mid;
                }
                const int pos = wtid + lo;
                mdest[pos] = d;
                msrc[pos] = lsrc[0][wtid];
                mref[pos] = lref[0][wtid];
            }
            if (wtid < VC) {
                const int d = ldest[1][wtid];
                int lo = 0, hi = VP;  // slot-0 entries with dest <= d
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (ldest[0][mid] <= d) lo = mid + 1;
                    else hi = mid;
                }
                const int pos = wtid + lo;
                mdest[pos] = d;
                msrc[pos] = lsrc[1][wtid];
                mref[pos] = lref[1][wtid];
            }
            wsync();
            const int V = VP + VC;
            int flag[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = 2 * wtid + h;
                flag[h] = r < V && (r == 0 || mdest[r] != mdest[r - 1]);
            }
            const int x = flag[0] + flag[1];
            int xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, xi, o);
                if (lane >= o) xi += y;
            }
            if (lane == 31) wtot[warp - 1] = xi;
            wsync();
            int before = 0, nsg = 0;
            for (int w2 = 0; w2 < LW; ++w2) {
                if (w2 < warp - 1) before += wtot[w2];
                nsg += wtot[w2];
            }
            int *lst = lists + L * LST;
            int *lsrcg = lst + 2, *lrefg = lsrcg + NE2, *lstart = lrefg + NE2, *ldestg = lstart + NE2 + 1;
            int idx = before + xi - x;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = 2 * wtid + h;
                if (r < V) {
                    lsrcg[r] = msrc[r];
                    lrefg[r] = mref[r];
                }
                if (flag[h]) {
                    lstart[idx] = r;
                    ldestg[idx] = mdest[r];
                    ++idx;
                }
            }
            if (wtid == 0) {
                lst[0] = V;
                lst[1] = nsg;
                lstart[nsg] = V;
            }
            wsync();  // the shared lists are reused by the next L
        }
    }
    // stale dots of the block at coordinate b1 (count nb1) against U copy R,
    // (chunk, coordinate) tasks: CTA `part` of `nparts` takes a contiguous
    // share (so every CTA gets some, and neighbouring warps take neighbouring
    // coordinates of one chunk, which mostly share the U column i_t: pairs
    // are in row order), one task per warp in turn, FP32 warp sums
    auto dots = [&](const float *R, int64_t b1, int nb1, double *out, int part, int nparts) {
        const int64_t ntask = (int64_t)nb1 * nch;
        const int64_t lo = ntask * part / nparts, hi = ntask * (part + 1) / nparts;
        for (int64_t task = lo + warp; task < hi; task += LT / 32) {
            const int c = (int)(task / nb1), t = (int)(task - (int64_t)c * nb1);
            const int64_t it_ = pi[b1 + t], jt = pj[b1 + t];
            const float *wr = W + jt * n;
            const float *uc = R + it_;
            const int64_t k0 = (int64_t)c * DCH, k1 = lmin(n, k0 + DCH);
            float acc = 0.f;
#pragma unroll 8
            for (int64_t k = k0 + lane; k < k1; k += 32) acc = fmaf(wr[k], uc[k * n], acc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) out[(int64_t)c * CD_B + t] = (double)acc;
        }
    };
    // prologue: dots of block 0 against copy 0 (both copies hold the initial U)
    dots(Ubuf0, 0, (int)lmin(CD_B, np), bvec, (int)blockIdx.x, (int)G);
    if (!grid_sync(gb, G, epoch, wc)) return;
    if (cc && tid == 32) {  // the matrices are complete after the barrier
        kcopy_issue(KIb, KallI, KB, &kbarI[0]);
        pendI0 = 1;
    }
    for (int64_t it = 0; it <= total; ++it) {
        const bool chain = it < total;
        if (cc) {
            if (!chain) break;
            const int64_t b0 = (it % nbatch) * CD_B;
            const int nb = (int)lmin(CD_B, np - b0);
            const bool need2 = it >= 1 && it + 1 < total;  // term of block it-1 on block it+1
            float *KI = KIb + (it & 1) * KS;
            // A. x, c and the threshold of block it (Delta is current in D: only
            //    this CTA writes it)
            {
                const double *bcur = bvec + (it & 1) * (int64_t)CD_MAX_CHUNKS * CD_B;
                for (int t = tid; t < CD_B; t += LT) {
                    if (t < nb) {
                        const double gv = g[b0 + t], av = aval[b0 + t], ia = inva[b0 + t];
                        const double d = D[b0 + t];
                        double b = gv;
                        if (nch <= 8) {
                            double v[8];
#pragma unroll
                            for (int r = 0; r < 8; ++r) v[r] = r < nch ? bcur[(int64_t)r * CD_B + t] : 0.0;
#pragma unroll
                            for (int r = 0; r < 8; ++r) b += v[r];
                        } else {
                            int c = 0;
                            for (; c + 8 <= nch; c += 8) {
                                double v[8];
#pragma unroll
                                for (int r = 0; r < 8; ++r) v[r] = bcur[(int64_t)(c + r) * CD_B + t];
#pragma unroll
                                for (int r = 0; r < 8; ++r) b += v[r];
                            }
                            for (; c < nch; ++c) b += bcur[(int64_t)c * CD_B + t];
                        }
                        const double cv = av + d;
                        xsh[t] = (float)(cv - b * ia) - xn[t];
                        csh[t] = (float)cv;
                        thsh[t] = (float)(lam * ia);
                        dold[t] = d;
                        aold[t] = av;
                    } else {
                        xsh[t] = csh[t] = thsh[t] = 0.f;
                    }
                }
            }
            __syncthreads();
            if (warp == 0) {
                // B. the chain
                if (lane == 0) kwait(&kbarI[it & 1], (it & 1) ? phI1 : phI0);
                __syncwarp();
                resolve_f32(KI, xsh, csh, thsh, nb, mush, zsh);
            } else {
                // copies for later: the next block's intra matrix (the other
                // buffer: its last reader was the previous chain) and this
                // block's +1 matrix (read in C)
                if (wtid == 0) {
                    if (it + 1 < total) {
                        kcopy_issue(KIb + ((it + 1) & 1) * KS, KallI + ((it + 1) % nbatch) * KS, KB,
                                    &kbarI[(it + 1) & 1]);
                        if ((it + 1) & 1) pendI1 = 1;
                        else pendI0 = 1;
                        kcopy_issue(K1, Kall1 + (it % nbatch) * KS, KB, &kbar1);
                        pend1 = 1;
                    }
                }
                // term of block it-1 (increments in mprev) on block it+1, from
                // the +2 matrix of block it-1 in global memory (coalesced rows)
                if (need2) {
                    const float *K2g = Kall2 + ((it - 1) % nbatch) * KS;
                    const int t = wtid & (CD_B - 1), h = wtid >> 7;
                    float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
                    for (int s2 = h * (CD_B / 2); s2 < (h + 1) * (CD_B / 2); s2 += 4) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) a[u] = fmaf(K2g[(s2 + u) * CD_B + t], mprev[s2 + u], a[u]);
                    }
                    xc2[h][t] = (a[0] + a[1]) + (a[2] + a[3]);
                }
            }
            if (it & 1) ++phI1;
            else ++phI0;
            if (wtid == 0) {
                if (it & 1) pendI1 = 0;
                else pendI0 = 0;
            }
            __syncthreads();
            // C. FP64 increments (exact zeros), written through to D
            if (tid < nb) {
                const double d0 = dold[tid];
                double m = 0.0, dn = d0;
                if (mush[tid] != 0.f) {
                    if (zsh[tid]) {
                        dn = -aold[tid];
                        m = dn - d0;
                    } else {
                        m = (double)mush[tid];
                        dn = d0 + m;
                    }
                }
                meff[tid] = m;
                D[b0 + tid] = dn;
            }
            __syncthreads();
            // the row-update multipliers of block it (entry e = 2t + k) for the
            // work CTAs, three generations by block index mod 3
            if (tid < NE) {
                const int e = tid, t = e >> 1;
                const float mu = t < nb ? (float)meff[t] : 0.f;
                gmu[(it % 3) * NE + e] = mu;
                if ((e & 1) == 0) mprev[t] = mu;
            }
            __syncthreads();
            // term of block it on block it+1; x of block it+1 loses both terms
            if (it + 1 < total) {
                if (tid == 0) kwait(&kbar1, ph1);
                ++ph1;
                if (wtid == 0) pend1 = 0;
                __syncthreads();
                if (tid < 2 * CD_B) {
                    const int t = tid & (CD_B - 1), h = tid >> 7;
                    float a0 = 0.f, a1 = 0.f;
                    for (int s2 = h * (CD_B / 2); s2 < (h + 1) * (CD_B / 2); s2 += 2) {
                        a0 = fmaf(K1[s2 * CD_B + t], mprev[s2], a0);
                        a1 = fmaf(K1[(s2 + 1) * CD_B + t], mprev[s2 + 1], a1);
                    }
                    x1[h][t] = a0 + a1;
                }
                __syncthreads();
                if (tid < CD_B)
                    xn[tid] = (need2 ? xc2[0][tid] + xc2[1][tid] : 0.f) + (x1[0][tid] + x1[1][tid]);
            }
        } else {
            // work CTA.  The merged list of blocks it-2 and it-1 and their
            // multipliers are loaded first (they land during the dots)
            const int64_t L = it == 0 ? -1 : (it == 1 ? nbatch : (it - 1) % nbatch);
            constexpr int PER = (NE2 + LT - 1) / LT;  // list words per thread and array
            int rs[PER], rr[PER], rst[PER], rd[PER], hdr0 = 0, hdr1 = 0;
            float rmu[PER];
            if (L >= 0) {
                const int *lst = lists + L * LST;
                const int *lsrcg = lst + 2, *lrefg = lsrcg + NE2, *lstart = lrefg + NE2, *ldestg = lstart + NE2 + 1;
                if (tid == 0) {
                    hdr0 = lst[0];
                    hdr1 = lst[1];
                }
#pragma unroll
                for (int u = 0; u < PER; ++u) {
                    const int r = tid + u * LT;
                    if (r < NE2) {
                        rs[u] = lsrcg[r];
                        rr[u] = lrefg[r];
                        rst[u] = lstart[r];
                        rd[u] = ldestg[r];
                        // multipliers: slot 0 = block it-2, slot 1 = block it-1
                        const int slot = r / NE, e = r - slot * NE;
                        const int64_t blk = it - 2 + slot;
                        rmu[u] = blk >= 0 ? gmu[(blk % 3) * NE + e] : 0.f;
                    }
                }
            }
            // stale dots of block it+1 against copy it mod 2 (all warps)
            if (it + 1 < total) {
                const int64_t nb0 = ((it + 1) % nbatch) * CD_B;
                dots((it & 1) ? Ubuf1 : Ubuf0, nb0, (int)lmin(CD_B, np - nb0),
                     bvec + ((it + 1) & 1) * (int64_t)CD_MAX_CHUNKS * CD_B, wb, GW);
            }
            if (L >= 0) {
#pragma unroll
                for (int u = 0; u < PER; ++u) {
                    const int r = tid + u * LT;
                    if (r < NE2) {
                        msrc[r] = rs[u];
                        mref[r] = rr[u];
                        seg_start[r] = rst[u];
                        seg_dest[r] = rd[u];
                        mutab[r] = rmu[u];
                    }
                }
                if (tid == 0) {
                    nv_s = hdr0;
                    nseg_s = hdr1;
                }
                __syncthreads();
                if (tid == 0) seg_start[nseg_s] = nv_s;
                __syncthreads();
                // apply to copy (it + 1) mod 2: items (segment, group of 4 columns
                // spaced by ncg) over the work CTAs, two per step with the loads first
                float *Y = (it & 1) ? Ubuf0 : Ubuf1;
                const int nseg = nseg_s;
                const int ncg = (int)((n + 3) / 4);
                const int items = nseg * ncg;
                const int nw = GW * LT;
                for (int q = wb * LT + tid; q < items; q += 2 * nw) {
                    const int qb = q + nw;
                    const bool hb = qb < items;
                    const int ka = q / ncg, ca = q - ka * ncg;
                    const int kb = hb ? qb / ncg : ka, cb = hb ? qb - kb * ncg : ca;
                    float *ura = Y + (int64_t)seg_dest[ka] * n, *urb = Y + (int64_t)seg_dest[kb] * n;
                    const int ea = seg_start[ka], eb = seg_start[kb];
                    const float ma = mutab[mref[ea]], mb = mutab[mref[eb]];
                    const float *wa = W + (int64_t)msrc[ea] * n, *wbr = W + (int64_t)msrc[eb] * n;
                    float ua[4], ub[4], va[4], vb[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int64_t col = ca + (int64_t)r * ncg, colb = cb + (int64_t)r * ncg;
                        ua[r] = col < n ? ura[col] : 0.f;
                        va[r] = col < n ? wa[col] : 0.f;
                        ub[r] = (hb && colb < n) ? urb[colb] : 0.f;
                        vb[r] = (hb && colb < n) ? wbr[colb] : 0.f;
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        ua[r] = fmaf(ma, va[r], ua[r]);
                        ub[r] = fmaf(mb, vb[r], ub[r]);
                    }
                    for (int e = ea + 1; e < seg_start[ka + 1]; ++e) {
                        const float m = mutab[mref[e]];
                        const float *wr = W + (int64_t)msrc[e] * n;
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const int64_t col = ca + (int64_t)r * ncg;
                            if (col < n) ua[r] = fmaf(m, wr[col], ua[r]);
                        }
                    }
                    if (hb)
                        for (int e = eb + 1; e < seg_start[kb + 1]; ++e) {
                            const float m = mutab[mref[e]];
                            const float *wr = W + (int64_t)msrc[e] * n;
#pragma unroll
                            for (int r = 0; r < 4; ++r) {
                                const int64_t col = cb + (int64_t)r * ncg;
                                if (col < n) ub[r] = fmaf(m, wr[col], ub[r]);
                            }
                        }
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int64_t col = ca + (int64_t)r * ncg, colb = cb + (int64_t)r * ncg;
                        if (col < n) ura[col] = ua[r];
                        if (hb && colb < n) urb[colb] = ub[r];
                    }
                }
            }
            if (!chain) break;
        }
        if (!grid_sync(gb, G, epoch, wc)) {
            drain();
            return;
        }
    }
}

// About 2 s of SM cycles unless a test has set a limit on the context.
WaitCfg wait_cfg(const Work &w) {
    return WaitCfg{w.dbg_wait_cycles > 0 ? w.dbg_wait_cycles : 4000000000ll,
                   w.dbg_wait_unreachable ? 1u : 0u};
}

OncePerDevice g_lag_once;
int g_lag_nsm[kMaxDevices], g_lag_occ[kMaxDevices];

OncePerDevice g_persist_once[4];
int g_persist_nsm[4][kMaxDevices], g_persist_occ[4][kMaxDevices];

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
    int dev = 0;
    cudaError_t ie = g_persist_once[which].run(dev, [&](int d) {
        cudaError_t e = cudaFuncSetAttribute(k_cd_persist<T, CT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kbytes);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&g_persist_nsm[which][d], cudaDevAttrMultiProcessorCount, d);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_persist_occ[which][d], k_cd_persist<T, CT>, RT,
                                                          kbytes);
        if (e != cudaSuccess) return e;
        return g_persist_occ[which][d] < 1 ? cudaErrorInvalidConfiguration : cudaSuccess;
    });
    if (ie != cudaSuccess) return ie;
    const int nsm = g_persist_nsm[which][dev], occ = g_persist_occ[which][dev];
    if (np <= 0 || nsweeps <= 0) return cudaSuccess;
    // enough CTAs for the row-update and dot phases, no more than co-resident
    int G = (int)lmax(4, lmin((int64_t)nsm * occ, (n + 7) / 8));
    // partial dots: ceil(n / DCH) x CD_B doubles, then the interaction matrix
    if ((n + DCH - 1) / DCH > CD_MAX_CHUNKS) return cudaErrorInvalidValue;
    double *bvec = w.cd_part;
    double *Kt = w.cd_part + (size_t)CD_MAX_CHUNKS * CD_B;
    static_assert(sizeof(GridBar) == 4 * sizeof(int), "barrier words");
    GridBar *gb = reinterpret_cast<GridBar *>(&w.sc->bar_count);
    cudaError_t e = cudaMemsetAsync(gb, 0, sizeof(GridBar), st);
    if (e != cudaSuccess) return e;
    const WaitCfg wc = wait_cfg(w);
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
                    (void *)&nsweeps, (void *)&bvec, (void *)&Kt, (void *)&Kall, (void *)&gb,
                    (void *)&wc};
    e = cudaLaunchCooperativeKernel((const void *)k_cd_persist<T, CT>, dim3(G), dim3(RT), args,
                                    kbytes, st);
    counted(1);
    path_hit(sizeof(CT) == 8 ? GLASSO_PATH_CD_CHAIN64 : GLASSO_PATH_CD_PERSIST32);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t cd_sweeps(const double *W, int64_t n, double lam, const int32_t *pi,
                      const int32_t *pj, int64_t np, const double *inva, const double *g,
                      const double *aval, int nsweeps, double *D, double *U, Work &w,
                      cudaStream_t st) {
    return cd_sweeps_t<double, double>(W, n, lam, pi, pj, np, inva, g, aval, nsweeps, D, U, w, st);
}

// FP32 sweep with the row updates off the serial path (k_cd_lag2); U2 is
// n x n FP32 scratch for the second copy of U.  Returns cudaErrorNotSupported
// when the interaction matrices of all blocks do not fit in n^2 doubles (the
// caller falls back to the one-copy sweep).
static cudaError_t cd_sweeps_lag(const float *W, int64_t n, double lam, const int32_t *pi,
                                 const int32_t *pj, int64_t np, const double *inva, const double *g,
                                 const double *aval, int nsweeps, double *D, float *U, float *U2,
                                 Work &w, cudaStream_t st) {
    if (n > (1 << 22) || (n + DCH - 1) / DCH > CD_MAX_CHUNKS) return cudaErrorNotSupported;
    const int64_t nbatch = (np + CD_B - 1) / CD_B;
    const size_t kb = (size_t)CD_B * CD_B * sizeof(float);
    const size_t kbytes = (size_t)(3 * nbatch) * kb;  // intra, +1, +2 matrices
    const size_t kneed = kbytes + (size_t)(nbatch + 1) * LST * sizeof(int);  // + merged lists
    if (kneed > (size_t)n * (size_t)n * sizeof(double)) return cudaErrorNotSupported;
    const size_t dyn = 3 * kb;  // two intra buffers and the +1 matrix
    int dev = 0;
    cudaError_t ie = g_lag_once.run(dev, [&](int d) {
        cudaError_t e = cudaFuncSetAttribute(k_cd_lag2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&g_lag_nsm[d], cudaDevAttrMultiProcessorCount, d);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_lag_occ[d], k_cd_lag2, LT, dyn);
        if (e != cudaSuccess) return e;
        return g_lag_occ[d] < 1 ? cudaErrorInvalidConfiguration : cudaSuccess;
    });
    if (ie != cudaSuccess) return ie;
    const int nsm = g_lag_nsm[dev], occ = g_lag_occ[dev];
    GridBar *gb = reinterpret_cast<GridBar *>(&w.sc->bar_count);
    cudaError_t e = cudaMemsetAsync(gb, 0, sizeof(GridBar), st);
    if (e != cudaSuccess) return e;
    const WaitCfg wc = wait_cfg(w);
    // both copies start as the current U
    e = cudaMemcpyAsync(U2, U, (size_t)n * (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    if (w.cap_cd_k < kneed) {
        const size_t want = std::min((size_t)n * (size_t)n * sizeof(double), std::max(kneed, 2 * w.cap_cd_k));
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
    float *Kall = reinterpret_cast<float *>(w.cd_k);
    double *bvec = w.cd_part;
    int *lists = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(w.cd_k) + kbytes);
    static_assert(3 * NE * sizeof(float) <= CD_B * CD_B * sizeof(double), "multiplier area");
    // row-update multipliers of the last three blocks, after the two
    // generations of partial dots
    float *gmu = reinterpret_cast<float *>(w.cd_part + (size_t)2 * CD_MAX_CHUNKS * CD_B);
    // the last pass (index total, no chain) writes copy (total + 1) mod 2: make that U
    const int64_t total = nbatch * (int64_t)nsweeps;
    float *b0 = ((total + 1) & 1) ? U2 : U, *b1 = ((total + 1) & 1) ? U : U2;
    const int G = (int)lmax(4, lmin((int64_t)nsm * occ, (n + 7) / 8));
    void *args[] = {(void *)&W, (void *)&b0, (void *)&b1, (void *)&n, (void *)&lam, (void *)&pi,
                    (void *)&pj, (void *)&np, (void *)&inva, (void *)&g, (void *)&aval, (void *)&D,
                    (void *)&nsweeps, (void *)&bvec, (void *)&Kall, (void *)&lists, (void *)&gmu, (void *)&gb,
                    (void *)&wc};
    e = cudaLaunchCooperativeKernel((const void *)k_cd_lag2, dim3(G), dim3(LT), args, dyn, st);
    counted(1);
    path_hit(GLASSO_PATH_CD_LAG2);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t cd_sweeps32(const float *W, int64_t n, double lam, const int32_t *pi,
                        const int32_t *pj, int64_t np, const double *inva, const double *g,
                        const double *aval, int nsweeps, double *D, float *U, Work &w,
                        bool chain64, cudaStream_t st, float *U2) {
    if (chain64)
        return cd_sweeps_t<float, double>(W, n, lam, pi, pj, np, inva, g, aval, nsweeps, D, U, w, st);
    if (U2 && np > 0 && nsweeps > 0) {
        cudaError_t e = cd_sweeps_lag(W, n, lam, pi, pj, np, inva, g, aval, nsweeps, D, U, U2, w, st);
        if (e != cudaErrorNotSupported) return e;
    }
    return cd_sweeps_t<float, float>(W, n, lam, pi, pj, np, inva, g, aval, nsweeps, D, U, w, st);
}

}  // namespace glx
