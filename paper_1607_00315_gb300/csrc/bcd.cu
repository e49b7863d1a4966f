// BCD-IC's line-search log det on the device (Section 6, Algorithm 2's
// update; eq. Schurs_lemma, eq. logdet_blocks, eq. Schurs_PDness).  For a
// block update A + alpha Delta whose Delta vanishes outside the rows and
// columns of the block I ("1"; "2" its complement):
//   log det(A + alpha Delta) = log det A_22 + log det(B_0 + alpha B_1 + alpha^2 B_2),
//   B_0 = A_11 - A_12 A_22^{-1} A_21,
//   B_1 = Delta_11 - Delta_12 A_22^{-1} A_21 - A_12 A_22^{-1} Delta_21,
//   B_2 = -Delta_12 A_22^{-1} Delta_21,
// and A + alpha Delta is positive definite iff A_22 and the small matrix are.
// The kernels here build the pieces; the FP64 factorisations and the inverse
// of A_22 are those of dense.cu (glasso_bcd_logdet in api.cu chains them).
#include "glasso_internal.h"

namespace glx {
namespace {

constexpr int BT = 256;

// Delta as a dense symmetric matrix from its pairs.  *bad = 1 when a pair
// with both indices outside the block carries a nonzero (not a block
// update), 2 when a pair index lies outside [0, n) (that pair is skipped).
__global__ void __launch_bounds__(BT) k_bcd_scatter(const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                                                   const double *__restrict__ D, int64_t np, int64_t n,
                                                   const uint8_t *__restrict__ inI, double *__restrict__ Dl,
                                                   int *bad) {
    const int64_t p = (int64_t)blockIdx.x * BT + threadIdx.x;
    if (p >= np) return;
    const int64_t i = pi[p], j = pj[p];
    if (i < 0 || j < 0 || i >= n || j >= n) {
        atomicExch(bad, 2);
        return;
    }
    const double d = D[p];
    if (!inI[i] && !inI[j] && d != 0.0) atomicExch(bad, 1);
    Dl[i * n + j] = d;
    Dl[j * n + i] = d;
}

// out (m x m, row-major) = A[idx, idx]
__global__ void __launch_bounds__(BT) k_bcd_gather(const double *__restrict__ A, int64_t n,
                                                  const int32_t *__restrict__ idx, int64_t m,
                                                  double *__restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * BT + threadIdx.x;
    if (e >= m * m) return;
    const int64_t a = e / m, c = e - a * m;
    out[e] = A[(int64_t)idx[a] * n + idx[c]];
}

// Column c of Y = A_22^{-1} A_21 and of Z = A_22^{-1} Delta_21 (stored at
// offset c m2), one entry per thread.
__global__ void __launch_bounds__(BT) k_bcd_solve(const double *__restrict__ Ainv, int64_t m2,
                                                 const double *__restrict__ A, const double *__restrict__ Dl,
                                                 int64_t n, const int32_t *__restrict__ idx1, int64_t m1,
                                                 const int32_t *__restrict__ idx2, double *__restrict__ Y,
                                                 double *__restrict__ Z) {
    const int64_t e = (int64_t)blockIdx.x * BT + threadIdx.x;
    if (e >= m2 * m1) return;
    const int64_t c = e / m2, k = e - c * m2;
    const int64_t col = idx1[c];
    double y = 0.0, z = 0.0;
    for (int64_t l = 0; l < m2; ++l) {
        const double w = Ainv[k * m2 + l];
        const int64_t r = (int64_t)idx2[l] * n + col;
        y = fma(w, A[r], y);
        z = fma(w, Dl[r], z);
    }
    Y[c * m2 + k] = y;
    Z[c * m2 + k] = z;
}

// M = B_0 + alpha B_1 + alpha^2 B_2 (m1 x m1), one entry per thread.
__global__ void __launch_bounds__(BT) k_bcd_assemble(const double *__restrict__ A, const double *__restrict__ Dl,
                                                    int64_t n, const int32_t *__restrict__ idx1, int64_t m1,
                                                    const int32_t *__restrict__ idx2, int64_t m2,
                                                    const double *__restrict__ Y, const double *__restrict__ Z,
                                                    double alpha, double *__restrict__ M) {
    const int64_t e = (int64_t)blockIdx.x * BT + threadIdx.x;
    if (e >= m1 * m1) return;
    const int64_t a = e / m1, c = e - a * m1;
    const int64_t ra = (int64_t)idx1[a] * n;
    double b0 = A[ra + idx1[c]], b1 = Dl[ra + idx1[c]], b2 = 0.0;
    for (int64_t k = 0; k < m2; ++k) {
        const int64_t col = idx2[k];
        const double a12 = A[ra + col], d12 = Dl[ra + col];
        const double y = Y[c * m2 + k], z = Z[c * m2 + k];
        b0 -= a12 * y;
        b1 -= d12 * y + a12 * z;
        b2 -= d12 * z;
    }
    M[e] = b0 + alpha * b1 + alpha * alpha * b2;
}

unsigned blocks_for(int64_t count) { return (unsigned)((count + BT - 1) / BT); }

}  // namespace

cudaError_t bcd_scatter(const int32_t *pi, const int32_t *pj, const double *D, int64_t np, int64_t n,
                        const uint8_t *inI, double *Dl, int *bad, cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    k_bcd_scatter<<<blocks_for(np), BT, 0, st>>>(pi, pj, D, np, n, inI, Dl, bad);
    counted(1);
    return cudaGetLastError();
}

cudaError_t bcd_gather(const double *A, int64_t n, const int32_t *idx, int64_t m, double *out, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_bcd_gather<<<blocks_for(m * m), BT, 0, st>>>(A, n, idx, m, out);
    counted(1);
    return cudaGetLastError();
}

cudaError_t bcd_solve(const double *Ainv, int64_t m2, const double *A, const double *Dl, int64_t n,
                      const int32_t *idx1, int64_t m1, const int32_t *idx2, double *Y, double *Z, cudaStream_t st) {
    if (m1 <= 0 || m2 <= 0) return cudaSuccess;
    k_bcd_solve<<<blocks_for(m2 * m1), BT, 0, st>>>(Ainv, m2, A, Dl, n, idx1, m1, idx2, Y, Z);
    counted(1);
    return cudaGetLastError();
}

cudaError_t bcd_assemble(const double *A, const double *Dl, int64_t n, const int32_t *idx1, int64_t m1,
                         const int32_t *idx2, int64_t m2, const double *Y, const double *Z, double alpha,
                         double *M, cudaStream_t st) {
    if (m1 <= 0) return cudaSuccess;
    k_bcd_assemble<<<blocks_for(m1 * m1), BT, 0, st>>>(A, Dl, n, idx1, m1, idx2, m2, Y, Z, alpha, M);
    counted(1);
    return cudaGetLastError();
}

}  // namespace glx
