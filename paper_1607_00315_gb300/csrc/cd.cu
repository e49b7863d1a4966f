// Coordinate-descent sweeps on the Newton LASSO of eq. Quad_MLE_l1_prior,
//   min_Delta tr(Delta G) + 1/2 tr(Delta W Delta W) + lambda ||A + Delta||_1,
// restricted to a pair list, keeping U = Delta W (Section 5.2: with W known
// the Hessian term costs O(|F| n)).  Coordinate (i, j) takes the exact 1-D
// minimiser of eq. 1d_l1, mu = -c + S_{lambda/a}(c - b/a), with
//   a = W_ij^2 + W_ii W_jj (W_ii^2 on the diagonal), c = A_ij + Delta_ij,
//   b = G_ij + (W Delta W)_ij,
// and the update U_i,: += mu W_j,:, U_j,: += mu W_i,: (one row on the diagonal).
//
// The sweep is a serial Gauss-Seidel chain.  It is run in blocks of B
// consecutive coordinates without changing its result (up to rounding):
//  1. dots (parallel): b0_t = G_t + W_{j_t,:} . U_{:,i_t} with U as it was
//     before the block ((W Delta W) is symmetric, so the j-row / i-column form
//     is used; pairs are sorted by i, so the U columns of a block are
//     contiguous).  The same launch computes the exact interaction
//     K[s][t] = (W E_s W)_{i_t j_t} = W_{i_t i_s} W_{j_s j_t} + W_{i_t j_s} W_{i_s j_t}
//     of an update of an earlier coordinate s on a later one t (one term when
//     s is diagonal).
//  2. resolve (one warp): for t = 0..B-1, b_t = b0_t + sum_{s<t} mu_s K[s][t],
//     mu_t from the closed form; the chain is a sequence of FMAs in shared
//     memory.  Delta is updated and the row updates are grouped by target row.
//  3. rows (parallel): each target row of U gets its updates in sweep order.
#include <math.h>

#include "glasso_internal.h"

namespace glx {
namespace {

constexpr int MAX_CHUNKS = 64;  // k-chunks of the dots
constexpr int NKB = 16;         // CTAs computing the interaction matrix
constexpr int RT = 256;         // threads of resolve / rows
constexpr int NE = 2 * CD_B;    // row-update entries per block
// cd_seg layout: [0] = #segments, [1 .. NE+1] segment starts, [NE+2 ..] targets
constexpr int SEG_START = 1;
constexpr int SEG_DEST = NE + 2;

template <typename CT>
__device__ __forceinline__ CT soft(CT x, CT t) {
    CT ax = fabs(x) - t;
    return ax > (CT)0 ? copysign(ax, x) : (CT)0;
}

// Stale dots, one CTA per coordinate t of the block: b0_t = G_t + W_{j_t,:} . U_{:,i_t},
// reduced in a fixed order (deterministic).  CTAs nb .. nb+NKB-1 compute the
// interaction matrix Kt[s][t] for sources s of their slice and all later t.
template <typename T>
__global__ void __launch_bounds__(CD_B) k_cd_dots(const T *__restrict__ W,
                                                  const T *__restrict__ U, int64_t n,
                                                  const int32_t *__restrict__ pi,
                                                  const int32_t *__restrict__ pj,
                                                  const double *__restrict__ g, int64_t b0, int nb,
                                                  double *__restrict__ bout,
                                                  double *__restrict__ Kt) {
    __shared__ int si[CD_B], sj[CD_B];
    __shared__ double red[CD_B];
    const int tid = threadIdx.x;
    const int c = blockIdx.x;
    if (c < nb) {
        const int64_t it = pi[b0 + c], jt = pj[b0 + c];
        const T *wr = W + jt * n;
        const T *uc = U + it;
        T acc = 0;
        for (int64_t k = tid; k < n; k += CD_B) acc = fma(wr[k], uc[k * n], acc);
        red[tid] = (double)acc;
        __syncthreads();
        for (int w = CD_B / 2; w > 0; w >>= 1) {
            if (tid < w) red[tid] += red[tid + w];
            __syncthreads();
        }
        if (tid == 0) bout[c] = g[b0 + c] + red[0];
        return;
    }
    if (tid < nb) {
        si[tid] = pi[b0 + tid];
        sj[tid] = pj[b0 + tid];
    }
    __syncthreads();
    const int kb = c - nb;
    const int per = CD_B / NKB;
    const int s0 = kb * per, s1 = min(nb, s0 + per);
    const int t = tid;
    if (t >= nb) return;
    const int64_t it = si[t], jt = sj[t];
    for (int s = s0; s < s1; ++s) {
        if (s >= t) break;
        const int64_t is = si[s], js = sj[s];
        double v = (double)W[it * n + is] * (double)W[js * n + jt];
        if (is != js) v = fma((double)W[it * n + js], (double)W[is * n + jt], v);
        Kt[s * CD_B + t] = v;
    }
}

// CT: arithmetic of the serial chain (FP64 for the FP64 path; FP32 for the
// mixed path, where one warp's FP64 issue rate would make the chain the
// sweep's critical path).  Delta itself is accumulated in FP64.
template <typename CT>
__global__ void __launch_bounds__(RT) k_cd_resolve(
    int64_t n, double lam, const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
    int64_t b0, int nb, const double *__restrict__ bin, const double *__restrict__ Kt,
    const double *__restrict__ inva, const double *__restrict__ g, const double *__restrict__ aval,
    double *__restrict__ D, int32_t *__restrict__ seg, int32_t *__restrict__ esrc,
    double *__restrict__ emu) {
    extern __shared__ __align__(16) unsigned char ks_raw[];
    CT *Ks = reinterpret_cast<CT *>(ks_raw);  // CD_B x CD_B, Ks[s * CD_B + t]
    __shared__ CT bsh[CD_B], csh[CD_B], ish[CD_B], mush[CD_B];
    __shared__ int zsh[CD_B];
    __shared__ double meff[CD_B];
    __shared__ int si[CD_B], sj[CD_B];
    __shared__ int edest[NE], evalid[NE];
    __shared__ int sdest[NE], ssrc[NE];
    __shared__ double smu[NE];
    __shared__ int nvalid_sh, nseg_sh;
    __shared__ int wtot[RT / 32];
    const int tid = threadIdx.x;
    (void)n;
    (void)g;
    if (tid < nb) {
        bsh[tid] = (CT)bin[tid];
        csh[tid] = (CT)(aval[b0 + tid] + D[b0 + tid]);
        ish[tid] = (CT)inva[b0 + tid];
        si[tid] = pi[b0 + tid];
        sj[tid] = pj[b0 + tid];
    }
    for (int q = tid; q < CD_B * CD_B; q += RT) {
        const int s = q / CD_B, t = q % CD_B;
        Ks[q] = (s < t && t < nb) ? (CT)Kt[q] : (CT)0;
    }
    __syncthreads();
    if (tid < 32) {
        const int lane = tid;
        for (int t = 0; t < nb; ++t) {
            if (lane == (t & 31)) {
                const CT c = csh[t], ia = ish[t];
                const CT z = soft(c - bsh[t] * ia, (CT)lam * ia);
                mush[t] = z - c;
                zsh[t] = (z == (CT)0);
            }
            __syncwarp();
            const CT mu = mush[t];
            if (mu != (CT)0) {
#pragma unroll
                for (int q = 0; q < CD_B / 32; ++q) {
                    const int s = lane + 32 * q;
                    if (s > t && s < nb) bsh[s] = fma(Ks[t * CD_B + s], mu, bsh[s]);
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    // Delta update (a zero from the shrinkage is written exactly:
    // A_ij + Delta_ij = 0) and the list of row updates (entry e = 2t + k)
    if (tid < nb) {
        double m = 0.0;
        if (mush[tid] != (CT)0) {
            const double d0 = D[b0 + tid];
            if (zsh[tid]) {
                const double dn = -aval[b0 + tid];
                D[b0 + tid] = dn;
                m = dn - d0;
            } else {
                m = (double)mush[tid];
                D[b0 + tid] = d0 + m;
            }
        }
        meff[tid] = m;
    }
    __syncthreads();
    for (int e = tid; e < NE; e += RT) {
        const int t = e >> 1, k = e & 1;
        int valid = 0, dst = 0;
        if (t < nb && meff[t] != 0.0) {
            if (k == 0) { valid = 1; dst = si[t]; }
            else if (si[t] != sj[t]) { valid = 1; dst = sj[t]; }
        }
        evalid[e] = valid;
        edest[e] = dst;
    }
    __syncthreads();
    // stable rank by target row
    for (int e = tid; e < NE; e += RT) {
        if (!evalid[e]) continue;
        const int d = edest[e];
        int r = 0;
        for (int f = 0; f < NE; ++f)
            r += evalid[f] && (edest[f] < d || (edest[f] == d && f < e));
        const int t = e >> 1;
        sdest[r] = d;
        ssrc[r] = (e & 1) ? si[t] : sj[t];
        smu[r] = meff[t];
    }
    if (tid == 0) {
        int v = 0;
        for (int e = 0; e < NE; ++e) v += evalid[e];
        nvalid_sh = v;
    }
    __syncthreads();
    const int V = nvalid_sh;
    // segment starts by a block scan of the start flags
    const int r = tid;  // RT == NE: one entry per thread
    const int start = (r < V) && (r == 0 || sdest[r] != sdest[r - 1]);
    int x = start;
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wtot[wid] = x;
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < RT / 32; ++w) {
        if (w < wid) before += wtot[w];
        total += wtot[w];
    }
    const int idx = before + x - start;
    if (start) {
        seg[SEG_START + idx] = r;
        seg[SEG_DEST + idx] = sdest[r];
    }
    if (r < V) {
        esrc[r] = ssrc[r];
        emu[r] = smu[r];
    }
    if (tid == 0) {
        nseg_sh = total;
        seg[0] = total;
        seg[SEG_START + total] = V;
    }
}

// Row updates: CTA (k, y) applies segment k's updates to columns
// [y * RCOLS, (y + 1) * RCOLS) of its target row, in sweep order.
constexpr int RCOLS = 512;
constexpr int RTH = 128;
template <typename T>
__global__ void __launch_bounds__(RTH) k_cd_rows(const T *__restrict__ W, T *__restrict__ U,
                                                 int64_t n, const int32_t *__restrict__ seg,
                                                 const int32_t *__restrict__ esrc,
                                                 const double *__restrict__ emu) {
    const int k = blockIdx.x;
    const int nseg = seg[0];
    if (k >= nseg) return;
    const int64_t dest = seg[SEG_DEST + k];
    const int e0 = seg[SEG_START + k], e1 = seg[SEG_START + k + 1];
    T *ur = U + dest * n;
    const int64_t c0 = (int64_t)blockIdx.y * RCOLS;
#pragma unroll
    for (int q = 0; q < RCOLS / RTH; ++q) {
        const int64_t col = c0 + threadIdx.x + q * RTH;
        if (col >= n) break;
        T u = ur[col];
        for (int e = e0; e < e1; ++e) u = fma((T)emu[e], W[(int64_t)esrc[e] * n + col], u);
        ur[col] = u;
    }
}

bool g_attr_done[2] = {false, false};

}  // namespace

template <typename T, typename CT>
static cudaError_t cd_sweeps_t(const T *W, int64_t n, double lam, const int32_t *pi,
                               const int32_t *pj, int64_t np, const double *inva, const double *g,
                               const double *aval, int nsweeps, double *D, T *U, Work &w,
                               cudaStream_t st) {
    static_assert(RT == NE, "one entry per thread in resolve");
    static_assert(CD_B % NKB == 0, "interaction split");
    const size_t kbytes = (size_t)CD_B * CD_B * sizeof(CT);
    const int which = sizeof(CT) == 8 ? 0 : 1;
    if (!g_attr_done[which]) {
        cudaError_t e = cudaFuncSetAttribute(k_cd_resolve<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kbytes);
        if (e != cudaSuccess) return e;
        g_attr_done[which] = true;
    }
    if (np <= 0) return cudaSuccess;
    double *bvec = w.cd_part;                           // CD_B stale dots
    double *Kt = w.cd_part + (size_t)MAX_CHUNKS * CD_B;  // CD_B x CD_B interactions
    const dim3 rgrid(NE, (unsigned)((n + RCOLS - 1) / RCOLS));
    for (int sw = 0; sw < nsweeps; ++sw) {
        for (int64_t b0 = 0; b0 < np; b0 += CD_B) {
            const int nb = (int)lmin(CD_B, np - b0);
            k_cd_dots<T><<<nb + NKB, CD_B, 0, st>>>(W, U, n, pi, pj, g, b0, nb, bvec, Kt);
            k_cd_resolve<CT><<<1, RT, kbytes, st>>>(n, lam, pi, pj, b0, nb, bvec, Kt, inva, g, aval,
                                                    D, w.cd_seg, w.cd_esrc, w.cd_emu);
            k_cd_rows<T><<<rgrid, RTH, 0, st>>>(W, U, n, w.cd_seg, w.cd_esrc, w.cd_emu);
            counted(3);
        }
    }
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
