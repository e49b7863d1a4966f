// Exact screening by connected components.
//
// Let the graph on {0..n-1} have an edge (i, j), i != j, where |S_ij| > lambda.
// The minimiser of eq. MLE_l1_prior is block diagonal over its connected
// components, and each block is the minimiser of the same problem on the
// block's principal sub-matrix of S.  Reason: assemble the blocks' minimisers
// into a block-diagonal A; then W = A^{-1} is block diagonal, and for a pair
// (i, j) in different components A_ij = 0 and |G_ij| = |S_ij - 0| <= lambda,
// which is the optimality condition of eq. subgradient1 at a zero entry.  All
// other conditions hold inside the blocks, and the minimiser is unique
// (Section 5).  An isolated vertex is a 1 x 1 block with the closed form
// A_ii = 1 / (S_ii + lambda).  The paper uses this separability in the
// divide-and-conquer comparison of Section 8 (blocks assumed there, exact
// here).
//
// Components are found by a lock-free union-find over the edges: a link
// always hangs the larger root under the smaller one (one compare-and-swap on
// the root's parent word), so every parent index is smaller than its child's
// and each component's final root is its smallest vertex, independent of the
// order in which the links land.
#include <math.h>

#include <algorithm>

#include "glasso_internal.h"

namespace glx {
namespace {

constexpr int CC_TPB = 256;

// Root of x.  Parent indices only decrease along a path, so the walk ends
// even on a stale read (a stale parent is still an ancestor).  Each visited
// vertex is pointed at its grandparent on the way (path splitting), which
// also keeps parent[v] <= v.  Parents are read through L2, since other SMs
// link roots meanwhile.
__device__ __forceinline__ int cc_find(int *parent, int x) {
    int p = __ldcg(parent + x);
    while (p != x) {
        const int g = __ldcg(parent + p);
        if (g != p) __stcg(parent + x, g);
        x = p;
        p = g;
    }
    return x;
}

__global__ void k_cc_init(int *__restrict__ parent, int *__restrict__ csize, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        parent[i] = (int)i;
        csize[i] = 0;
    }
}

// One row of the upper triangle per block step, coalesced along the row; each
// edge links the two roots.  A failed compare-and-swap means the larger root
// was linked meanwhile (at most n - 1 links happen in all, and the retried
// roots strictly decrease), so 2n + 64 attempts per edge cannot be exceeded;
// the bound only guards against a broken invariant, and sets *err.
__global__ void k_cc_hook(const double *__restrict__ S, int64_t n, double lam, int *parent,
                          int *err) {
    const int limit = 2 * (int)n + 64;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const double *row = S + i * n;
        for (int64_t j = i + 1 + threadIdx.x; j < n; j += blockDim.x) {
            if (!(fabs(row[j]) > lam)) continue;
            int a = cc_find(parent, (int)i), b = cc_find(parent, (int)j);
            for (int it = 0; a != b; ++it) {
                if (it >= limit) {
                    atomicExch(err, 1);
                    break;
                }
                if (a > b) {
                    const int t = a;
                    a = b;
                    b = t;
                }
                const int old = atomicCAS(parent + b, b, a);
                if (old == b) break;
                a = cc_find(parent, a);
                b = cc_find(parent, old);
            }
        }
    }
}

__global__ void k_cc_final(int *parent, int64_t n, int32_t *__restrict__ comp, int *csize) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = cc_find(parent, (int)i);
        comp[i] = r;
        atomicAdd(csize + r, 1);
    }
}

// Isolated vertices: the closed form on the diagonal of A (and of W); every
// diagonal entry of S is copied out for the host's objective sums.
__global__ void k_screen_diag(const double *__restrict__ S, int64_t n, double lam,
                              const int32_t *__restrict__ comp, const int *__restrict__ csize,
                              double *__restrict__ A, double *__restrict__ W,
                              double *__restrict__ diag, int *err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double s = S[i * n + i];
        diag[i] = s;
        if (csize[comp[i]] != 1) continue;
        const double d = s + lam;
        if (!(d > 0.0)) atomicExch(err, 1);
        A[i * n + i] = 1.0 / d;
        if (W) W[i * n + i] = d;
    }
}

// dst (nb x nb, row stride nb) = src[idx, idx] (row stride n); one dst row per
// block step.
__global__ void k_gather_block(const double *__restrict__ src, int64_t n,
                               const int32_t *__restrict__ idx, int64_t nb,
                               double *__restrict__ dst) {
    for (int64_t a = blockIdx.x; a < nb; a += gridDim.x) {
        const double *row = src + (int64_t)idx[a] * n;
        for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) dst[a * nb + b] = row[idx[b]];
    }
}

// dst[idx, idx] (row stride n) = src (nb x nb, row stride nb).
__global__ void k_scatter_block(const double *__restrict__ src, int64_t nb,
                                const int32_t *__restrict__ idx, int64_t n,
                                double *__restrict__ dst) {
    for (int64_t a = blockIdx.x; a < nb; a += gridDim.x) {
        double *row = dst + (int64_t)idx[a] * n;
        for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) row[idx[b]] = src[a * nb + b];
    }
}

unsigned grid_rows(int64_t rows) { return (unsigned)std::min<int64_t>(std::max<int64_t>(rows, 1), 152 * 8); }
unsigned grid_elems(int64_t k) {
    return (unsigned)std::min<int64_t>(std::max<int64_t>((k + CC_TPB - 1) / CC_TPB, 1), 152 * 8);
}

}  // namespace

cudaError_t components(const double *S, int64_t n, double lam, int *parent, int32_t *comp,
                       int *csize, int *err, cudaStream_t st) {
    if (n < 1 || n > (int64_t)1 << 30) return cudaErrorInvalidValue;
    k_cc_init<<<grid_elems(n), CC_TPB, 0, st>>>(parent, csize, n);
    k_cc_hook<<<grid_rows(n), CC_TPB, 0, st>>>(S, n, lam, parent, err);
    k_cc_final<<<grid_elems(n), CC_TPB, 0, st>>>(parent, n, comp, csize);
    counted(3);
    return cudaGetLastError();
}

cudaError_t screen_diag(const double *S, int64_t n, double lam, const int32_t *comp, const int *csize,
                        double *A, double *W, double *diag, int *err, cudaStream_t st) {
    k_screen_diag<<<grid_elems(n), CC_TPB, 0, st>>>(S, n, lam, comp, csize, A, W, diag, err);
    counted(1);
    return cudaGetLastError();
}

cudaError_t gather_block(const double *src, int64_t n, const int32_t *idx, int64_t nb, double *dst,
                         cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    k_gather_block<<<grid_rows(nb), CC_TPB, 0, st>>>(src, n, idx, nb, dst);
    counted(1);
    return cudaGetLastError();
}

cudaError_t scatter_block(const double *src, int64_t nb, const int32_t *idx, int64_t n, double *dst,
                          cudaStream_t st) {
    if (nb <= 0) return cudaSuccess;
    k_scatter_block<<<grid_rows(nb), CC_TPB, 0, st>>>(src, nb, idx, n, dst);
    counted(1);
    return cudaGetLastError();
}

}  // namespace glx
