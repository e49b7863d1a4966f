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
// The barrier is a counter plus generation word in global memory; every wait
// is bounded (2 s, globaltimer) and sets an error word read by the host.
struct GridBar {
    unsigned count;
    unsigned gen;
    int err;
    int pad;
};

__device__ __forceinline__ unsigned long long cd_gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool grid_sync(GridBar *gb, unsigned nblocks) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &gb->gen;
        volatile int *verr = &gb->err;
        const unsigned g0 = *vgen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(&gb->count, 1u) == nblocks - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            const unsigned long long t0 = cd_gtimer();
            while (*vgen == g0) {
                if (*verr || cd_gtimer() - t0 > 2000000000ull) {
                    ok = 0;
                    atomicExch(&gb->err, 1);
                    break;
                }
            }
        }
        __threadfence();
        ok_s = ok && !*verr;
    }
    __syncthreads();
    return ok_s != 0;
}

template <typename T, typename CT>
__global__ void __launch_bounds__(RT, 1) k_cd_persist(
    const T *__restrict__ W, T *__restrict__ U, int64_t n, double lam,
    const int32_t *__restrict__ pi, const int32_t *__restrict__ pj, int64_t np,
    const double *__restrict__ inva, const double *__restrict__ g, const double *__restrict__ aval,
    double *__restrict__ D, int nsweeps, double *__restrict__ bvec, double *__restrict__ Kt,
    GridBar *gb) {
    extern __shared__ __align__(16) unsigned char ks_raw[];
    CT *Ks = reinterpret_cast<CT *>(ks_raw);  // Ks[s * CD_B + t]
    __shared__ CT bsh[CD_B], csh[CD_B], ish[CD_B], mush[CD_B];
    __shared__ int zsh[CD_B];
    __shared__ double meff[CD_B], dnew[CD_B];
    __shared__ int si[CD_B], sj[CD_B];
    __shared__ unsigned skey[NE];
    __shared__ int sdest[NE], ssrc[NE];
    __shared__ double smu[NE];
    __shared__ int seg_start[NE + 1], seg_dest[NE];
    __shared__ int nseg_s, wtot[RT / 32];
    const unsigned G = gridDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t gthread = (int64_t)blockIdx.x * RT + tid, nthreads = (int64_t)G * RT;
    const int64_t gwarp = (int64_t)blockIdx.x * (RT / 32) + warp, nwarps = (int64_t)G * (RT / 32);
    const int64_t nbatch = (np + CD_B - 1) / CD_B;
    const int64_t total = nbatch * nsweeps;
    int64_t prev_b0 = -1;
    int prev_nb = 0;
    if (tid == 0) nseg_s = 0;
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
                    const T m = (T)smu[e];
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
        if (!grid_sync(gb, G)) return;
        if (blockIdx.x == 0 && prev_b0 >= 0)
            for (int t = tid; t < prev_nb; t += RT) D[prev_b0 + t] = dnew[t];
        const int64_t b0 = (it % nbatch) * CD_B;
        const int nb = (int)lmin(CD_B, np - b0);
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
            double a = (double)acc;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) bvec[(int64_t)c * CD_B + t] = a;
        }
        CT *Ktc = reinterpret_cast<CT *>(Kt);
        for (int q = (int)gthread; q < nb * nb; q += (int)nthreads) {
            const int s = q / nb, t = q - s * nb;
            if (s < t) {
                const int64_t is = pi[b0 + s], js = pj[b0 + s], it2 = pi[b0 + t], jt = pj[b0 + t];
                double v = (double)W[it2 * n + is] * (double)W[js * n + jt];
                if (is != js) v = fma((double)W[it2 * n + js], (double)W[is * n + jt], v);
                Ktc[s * CD_B + t] = (CT)v;
            }
        }
        if (!grid_sync(gb, G)) return;
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
        }
        {
            // the interaction matrix as 16-byte vectors, eight independent loads
            // in flight per thread (entries with s >= t or t >= nb are ignored by
            // the chain, whatever they hold)
            constexpr int VEC = 16 / sizeof(CT);
            const uint4 *src = reinterpret_cast<const uint4 *>(Kt);
            uint4 *dst = reinterpret_cast<uint4 *>(Ks);
            constexpr int NV = CD_B * CD_B / VEC;
#pragma unroll 8
            for (int q = tid; q < NV; q += RT) dst[q] = src[q];
        }
        __syncthreads();
        if (tid < 32) {
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
        for (int e = tid; e < NE; e += RT) {
            const int t = e >> 1, k = e & 1;
            unsigned key = 0xFFFFFFFFu;
            if (t < nb && meff[t] != 0.0) {
                if (k == 0) key = ((unsigned)si[t] << 9) | (unsigned)e;
                else if (si[t] != sj[t]) key = ((unsigned)sj[t] << 9) | (unsigned)e;
            }
            skey[e] = key;
        }
        __syncthreads();
        for (int size = 2; size <= NE; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                const int e = tid, pr = e ^ stride;
                if (pr > e) {
                    const bool up = (e & size) == 0;
                    const unsigned a = skey[e], b = skey[pr];
                    if ((a > b) == up) {
                        skey[e] = b;
                        skey[pr] = a;
                    }
                }
                __syncthreads();
            }
        }
        int V = 0;
        {
            const unsigned kk = skey[tid];
            const int valid = kk != 0xFFFFFFFFu;
            if (valid) {
                const int e = (int)(kk & 511u), t = e >> 1;
                sdest[tid] = (int)(kk >> 9);
                ssrc[tid] = (e & 1) ? si[t] : sj[t];
                smu[tid] = meff[t];
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
    void *args[] = {(void *)&W, (void *)&U, (void *)&n, (void *)&lam, (void *)&pi, (void *)&pj,
                    (void *)&np, (void *)&inva, (void *)&g, (void *)&aval, (void *)&D,
                    (void *)&nsweeps, (void *)&bvec, (void *)&Kt, (void *)&gb};
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
