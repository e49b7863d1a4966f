// Internal declarations shared by the CUDA translation units of the solver.
// Everything here is private to the shared library; the public surface is
// include/glasso.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>

#include "glasso.h"

namespace glx {

// One-time set-up per device (kernel attributes, occupancy), thread-safe:
// host threads of the serving slots may enter a launcher together, and a
// process may drive several devices.  init(dev) runs once per device; its
// status is returned to every caller.
constexpr int kMaxDevices = 64;
struct OncePerDevice {
    std::once_flag flag[kMaxDevices];
    cudaError_t status[kMaxDevices] = {};
    template <typename F>
    cudaError_t run(int &dev, F init) {
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
        std::call_once(flag[dev], [&] { status[dev] = init(dev); });
        return status[dev];
    }
};

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation runs its prologue while its predecessor finishes; it must
// pass pdl_wait() (the predecessor complete, its writes visible) before it
// reads anything the predecessor wrote.  pdl_trigger() lets the successor
// start its own prologue.  Both are no-ops for a normal launch.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#endif


__host__ __device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t lmax(int64_t a, int64_t b) { return a > b ? a : b; }

// Number of kernels this library has launched (all contexts); read through
// glasso_profile.kernels.
extern std::atomic<long long> g_launches;
inline void counted(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Counters of the solver's code paths (all contexts), read through
// glasso_profile.paths; indexes are the GLASSO_PATH_* values of glasso.h.
extern std::atomic<long long> g_paths[GLASSO_PATHS];
inline void path_hit(int k, long long v = 1) { g_paths[k].fetch_add(v, std::memory_order_relaxed); }

// Column / row block of the dense FP64 kernels (Cholesky panel width, tile edge).
constexpr int NB = 32;
// Coordinates resolved together by one blocked CD step (see cd.cu).
constexpr int CD_B = 128;
// Maximum number of 256-column chunks of the CD dot products (n <= 65536).
constexpr int CD_MAX_CHUNKS = 256;

// Device-side scalar results of the reduction kernels (one struct per context).
struct DevScalars {
    // full free-set scan (level 0)
    long long count;      // free pairs written
    double kkt_sum;       // sum_ij |min-norm subgradient|
    double kkt_max;       // max_ij |min-norm subgradient|
    double trSA;          // sum_ij S_ij A_ij
    double l1;            // sum_ij |A_ij|
    long long nnz;        // #{A_ij != 0}
    // Cholesky
    int info;             // 0 or first failing pivot + 1
    int pad0;
    double logdet;
    // line search
    double delta;         // tr(G Delta) + lambda (||A + Delta||_1 - ||A||_1)
    double trSD;          // tr(S Delta)
    double dl1;           // ||A + alpha Delta||_1 - ||A||_1 at the trial alpha
    int moved;            // any Delta_p != 0
    int levels;           // hierarchy levels L
    long long nsupp;
    // mixed precision
    double ns_max;        // max |I - A W|
    double ns_fro2;       // ||I - A W||_F^2
    double t1;            // tr(W Delta)
    double t2;            // tr((W Delta)^2)
    double t3, t4, t5, t6;  // tr((W Delta)^k), k = 3..6
    int err;              // device-side error flag (NaN input, bad diagonal)
    int bad_sym;          // input symmetry check failed
    int tc_err;           // tensor-core GEMM: a bounded wait expired (code)
    unsigned res_done;    // residual: CTAs finished (the last one reduces, then resets it)
    // grid barrier of the persistent CD sweep: count, generation, error, pad
    unsigned bar_count;
    unsigned bar_gen;
    int bar_err;
    int cc_err;           // component labelling: a retry bound was exceeded
    unsigned long long smax_bits;  // max_{i != j} |S_ij| as the bits of a non-negative double
    unsigned scan_done;   // free-set sums: CTAs finished (the last one reduces, then resets it)
    unsigned pad1;
};

// Per-context device workspace, sized for n <= cap_n.
struct Work {
    int64_t cap_n = 0;
    int64_t cap_pairs = 0;
    double *S = nullptr, *A = nullptr, *L = nullptr, *T = nullptr, *W = nullptr, *U = nullptr;
    double *Xin = nullptr;       // centred FP64 copy of X (m x n) and its mean (n)
    int64_t cap_x = 0;
    char *Xraw = nullptr;        // host samples copied to the device as given
    int64_t cap_xraw = 0;
    // pair lists
    int32_t *fi = nullptr, *fj = nullptr;  // previous fine free set F_k
    double *fabsg = nullptr;               // |G| on F_k
    uint8_t *ftag = nullptr, *fsupp = nullptr;
    int32_t *pi = nullptr, *pj = nullptr;  // current relaxation's free set
    double *pabsg = nullptr;
    double *D = nullptr;                   // Delta on pairs
    double *p_inva = nullptr, *p_g = nullptr, *p_a = nullptr, *p_s = nullptr;
    // scan / compaction scratch
    uint32_t *mask = nullptr;              // n x ceil(n/32) bit masks
    long long *rowcnt = nullptr;           // n + 1
    double *rowred = nullptr;              // n x 6 partial sums
    uint8_t *flags = nullptr;              // cap_pairs
    long long *blkcnt = nullptr;           // blocks of the compaction
    int64_t cap_blk = 0;
    double *redbuf = nullptr;              // generic reduction partials
    int64_t cap_red = 0;
    // CD scratch
    double *cd_part = nullptr;             // 2 x CD_MAX_CHUNKS x CD_B partial dots, then CD_B^2 K
    float *fa = nullptr;                   // 4 x n x tc_pad(n) FP32: matrix, X, Xt, scratch of cholinv_tc
    unsigned char *cd_k = nullptr;         // interaction matrices of all CD blocks (grown on demand)
    size_t cap_cd_k = 0;
    double *xd = nullptr;                  // 2 x 32 x 32: inverses of Cholesky diagonal blocks
    double *ldiag = nullptr;               // n: FP64 diagonal of the last factor
    // mixed precision: CSR of A and reduction partials
    int64_t cap_mixed = 0;
    long long *csr_ptr = nullptr;
    int32_t *csr_col = nullptr;
    double *csr_val = nullptr;
    double *part = nullptr;
    int64_t cap_part = 0;
    float *Wp = nullptr, *Qp = nullptr;    // padded FP32 operands of the tensor-core GEMM
    float *U2p = nullptr, *U3p = nullptr;  // padded U^2, U^3 of the log-det series
    float *Xt = nullptr;                   // padded X^T for S on the tensor cores
    int64_t cap_xt = 0;
    DevScalars *sc = nullptr;              // device scalars
    DevScalars *sc_host = nullptr;         // pinned mirror
    // a lower-priority stream and two events for the factorisation's off-path
    // GEMMs (created on first use)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    // screening: the full S, A, W and A0 while a sub-problem occupies S .. U,
    // the component labels and the sub-problem's vertex list
    int64_t cap_scr = 0, cap_cc = 0;
    double *scr_S = nullptr, *scr_A = nullptr, *scr_W = nullptr, *scr_A0 = nullptr;
    double *scr_diag = nullptr;
    int *cc_parent = nullptr, *cc_size = nullptr;
    int32_t *cc_comp = nullptr, *scr_idx = nullptr;
    // PCD-CG scratch (pcd.cu): pair vectors and CSR of the pairs, grown on demand
    unsigned char *pcd_vec = nullptr;
    int64_t pcd_cap_np = 0;
    int *pcd_rows = nullptr;
    int64_t pcd_cap_n = 0;
    // fault injection for tests of the error paths (glasso_set_debug)
    long long dbg_wait_cycles = 0;  // CD grid-barrier wait limit in SM cycles (0: about 2 s)
    int dbg_wait_unreachable = 0;   // the barrier waits for one arrival more than the grid holds
    int dbg_ls_reject = 0;          // every line-search trial is rejected
    int dbg_dag_tiles = 0;          // largest task-graph block in tiles (0: default, 1: none)
    int dag_share = 1;              // a task-graph launch takes at most 1 / dag_share of the SMs
                                    // (the serving slots' solves run concurrently)
};

}  // namespace glx

struct glasso_ctx {
    int device = 0;
    int precision = GLASSO_FP64;
    size_t budget = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    glx::Work w;
    std::string last_error;
    void *serve = nullptr;  // serving state (api.cu)
    void *prof = nullptr;   // kernel-class timing (api.cu)
};

namespace glx {

// ---- launchers (dense.cu) ----
cudaError_t form_S(const void *X, int dtype, int64_t m, int64_t n, int center, double *S,
                   double *mu_scratch, cudaStream_t st);
// In-place blocked Cholesky of the lower triangle; writes sc->info and sc->logdet.
// xd: scratch of 2 * NB * NB elements (inverses of the diagonal blocks);
// ldiag: n doubles receiving the FP64 diagonal of L (the log-det reads it).
cudaError_t potrf(double *A, int64_t n, double *xd, double *ldiag, DevScalars *sc, cudaStream_t st);
// Same factorisation in FP32 storage and arithmetic, diagonal blocks in FP64.
cudaError_t potrf32(float *A, int64_t n, float *xd, double *ldiag, DevScalars *sc, cudaStream_t st);
// W = L^{-T} L^{-1}; X (n x n) and Tw (n x n) are scratch.
cudaError_t inverse(const double *L, int64_t n, double *W, double *X, double *Tw, cudaStream_t st);
cudaError_t inverse32(const float *L, int64_t n, float *W, float *X, float *Tw, cudaStream_t st);

// ---- launchers (scan.cu) ----
// Full level-0 scan: free set (pi, pj, absg) and the sums of DevScalars.
// mode 0: condition A != 0 or |S - W| > lambda; mode 1: A != 0 or |S| > lambda
// (the initial free set of Section 7's footnote).
cudaError_t scan_full(const double *S, const double *W, const double *A, int64_t n, double lam,
                      int mode, Work &w, int32_t *oi, int32_t *oj, double *oabsg, DevScalars *sc,
                      cudaStream_t st);
// Candidate scan: keep candidates p with (tag == NULL or tag[p] >= level) that
// are free; writes count to sc->count.
cudaError_t scan_cand(const double *S, const double *W, const double *A, int64_t n, double lam,
                      const int32_t *ci, const int32_t *cj, const uint8_t *tag, int level,
                      int64_t ncand, Work &w, int32_t *oi, int32_t *oj, double *oabsg,
                      DevScalars *sc, cudaStream_t st);
cudaError_t support_flags(const double *A, int64_t n, const int32_t *fi, const int32_t *fj,
                          int64_t nf, uint8_t *flag, cudaStream_t st);
cudaError_t init_diag(const double *S, int64_t n, double lam, double *A, DevScalars *sc,
                      cudaStream_t st);
// sc->smax_bits = the bits of max_{i < j} |S_ij| (0 for n = 1)
cudaError_t offdiag_absmax(const double *S, int64_t n, DevScalars *sc, cudaStream_t st);

// ---- screening (screen.cu) ----
// Connected components of {(i, j): i != j, |S_ij| > lambda}: comp[i] = the
// smallest vertex of i's component, csize[r] = the size of the component
// whose smallest vertex is r (0 elsewhere).  parent, csize: n ints of scratch.
cudaError_t components(const double *S, int64_t n, double lam, int *parent, int32_t *comp,
                       int *csize, int *err, cudaStream_t st);
// For each isolated vertex i: A_ii = 1/(S_ii + lambda) and W_ii = S_ii + lambda
// (W may be NULL); diag[i] = S_ii for every i; *err = 1 if some S_ii + lambda <= 0.
cudaError_t screen_diag(const double *S, int64_t n, double lam, const int32_t *comp, const int *csize,
                        double *A, double *W, double *diag, int *err, cudaStream_t st);
// dst (nb x nb) = src[idx, idx] and back; idx holds nb distinct indices < n.
cudaError_t gather_block(const double *src, int64_t n, const int32_t *idx, int64_t nb, double *dst,
                         cudaStream_t st);
cudaError_t scatter_block(const double *src, int64_t nb, const int32_t *idx, int64_t n, double *dst,
                          cudaStream_t st);
// per-pair data for the CD sweep
cudaError_t pair_prep(const double *S, const double *W, const double *A, int64_t n, double lam,
                      const int32_t *pi, const int32_t *pj, int64_t np, double *inva, double *g,
                      double *aval, double *sval, cudaStream_t st);
// line search pieces
cudaError_t ls_delta(const double *g, const double *aval, const double *sval, const double *D,
                     const int32_t *pi, const int32_t *pj, int64_t np, double lam, Work &w,
                     DevScalars *sc, cudaStream_t st);
cudaError_t ls_build_trial(const double *A, double *T, int64_t n, const int32_t *pi,
                           const int32_t *pj, const double *aval, const double *D, int64_t np,
                           double alpha, cudaStream_t st);
cudaError_t ls_dl1(const double *aval, const double *D, const int32_t *pi, const int32_t *pj,
                   int64_t np, double alpha, Work &w, DevScalars *sc, cudaStream_t st);
cudaError_t ls_apply(double *A, int64_t n, const int32_t *pi, const int32_t *pj,
                     const double *aval, const double *D, int64_t np, double alpha,
                     cudaStream_t st);

// ---- launchers (hier.cu) ----
cudaError_t hierarchy(const double *absg, const uint8_t *insupp, int64_t nf, uint8_t *tag,
                      DevScalars *sc, cudaStream_t st);

// ---- launchers (mixed.cu) ----
cudaError_t build_csr(const double *A, int64_t n, long long *ptr, int32_t *col, double *val,
                      cudaStream_t st);
cudaError_t residual(const long long *ptr, const int32_t *col, const double *val, const float *Whi,
                     const float *Wlo, int64_t n, float *R32, double *rowstat, DevScalars *sc,
                     cudaStream_t st);
cudaError_t series_terms(const double *W64, int64_t n, const int32_t *pi, const int32_t *pj,
                         const double *D, int64_t np, const float *U32, double *part, int64_t cap,
                         DevScalars *sc, cudaStream_t st);
cudaError_t series_high(const float *U32, int64_t n, float *Up, float *Ut, float *U2, float *U3,
                        double *part, int64_t cap, DevScalars *sc, cudaStream_t st);
cudaError_t to_f32(const double *x, float *y, int64_t m, cudaStream_t st);
cudaError_t split64(const double *W, float *hi, float *lo, int64_t m, cudaStream_t st);
cudaError_t join64(const float *hi, const float *lo, double *W, int64_t m, cudaStream_t st);
cudaError_t to_f64(const float *x, double *y, int64_t m, cudaStream_t st);
cudaError_t trial32(const double *A, float *T, int64_t n, int64_t ldT, const int32_t *pi,
                    const int32_t *pj, const double *aval, const double *D, int64_t np, double alpha,
                    cudaStream_t st);
cudaError_t diag_inverse(const double *A, int64_t n, double *W64, double *logs, DevScalars *sc,
                         cudaStream_t st);

// ---- launchers (tc.cu) ----
int64_t tc_pad(int64_t n);
// FP32 factorisation and inverse on the tensor cores (split TF32): see cholinv_tc.cu
cudaError_t chol_leaf32(const float *A, int64_t ld, int64_t o, int s, float *X, float *Xt, double *ldiag,
                        DevScalars *sc, cudaStream_t st);
cudaError_t logdet_from_diag(const double *ldiag, int64_t n, DevScalars *sc, cudaStream_t st);
cudaError_t cholinv_tc(float *A, int64_t n, int64_t ld, float *X, float *Xt, float *Z, double *ldiag,
                       DevScalars *sc, cudaStream_t st, cudaStream_t side = nullptr,
                       cudaEvent_t ev_a = nullptr, cudaEvent_t ev_b = nullptr, int dag_tiles = 0,
                       int dag_share = 1);
// one persistent task-graph launch for a diagonal block (chol_dag.cu); a
// block fits when 128 < s <= max_tiles * 128 (max_tiles 0: the default 32)
bool chol_dag_fits(int64_t s, int max_tiles = 0);
cudaError_t chol_dag(float *A, int64_t ld, int64_t o, int64_t s, float *X, float *Xt, double *ldiag,
                     unsigned *scratch, DevScalars *sc, cudaStream_t st, long long wait_cycles = 0,
                     int share = 1);
cudaError_t lauum_tc(const float *Xt, int64_t n, int64_t ld, float *W, int64_t ldw, DevScalars *sc,
                     cudaStream_t st);
cudaError_t gemm_nt_split(const float *P, const float *Q, int64_t n, int64_t ld, float *C, int *err,
                          cudaStream_t st);
cudaError_t syrk_split(const float *Xt, int64_t n, int64_t m, int64_t ldx, double scale, double *S,
                       int *err, cudaStream_t st);
cudaError_t ns_gemm_tc(const float *Whi, float *Whi_next, float *Wlo, const float *R32, int64_t n,
                       float *Wp, float *Qp, int *err, cudaStream_t st);
cudaError_t syrk_tc(const void *X, int dtype, int64_t m, int64_t n, const double *mu, double *S,
                    float *Xt, int *err, cudaStream_t st);
cudaError_t pad_and_transpose(const float *U, int64_t n, float *Up, float *Ut, cudaStream_t st);

// ---- launchers (cd.cu) ----
cudaError_t cd_sweeps(const double *W, int64_t n, double lam, const int32_t *pi,
                      const int32_t *pj, int64_t np, const double *inva, const double *g,
                      const double *aval, int nsweeps, double *D, double *U, Work &w,
                      cudaStream_t st);
// PCD-CG Newton-direction solver on the pair list (pcd.cu): W, U, Vt n x n
// (Vt scratch); D on the pairs in/out (d_nonzero: D may be nonzero on entry);
// U = Delta W on return; *iters_done (host, optional; synchronises).
cudaError_t pcd(const double *W, int64_t n, double lam, const int32_t *pi, const int32_t *pj, int64_t np,
                const double *inva, const double *g, const double *aval, int iters, int cg, double rtol,
                double *D, double *U, double *Vt, bool d_nonzero, Work &w, cudaStream_t st, int *iters_done);
cudaError_t pcd32(const float *W, int64_t n, double lam, const int32_t *pi, const int32_t *pj, int64_t np,
                  const double *inva, const double *g, const double *aval, int iters, int cg, double rtol,
                  double *D, float *U, float *Vt, bool d_nonzero, Work &w, cudaStream_t st, int *iters_done);
cudaError_t cd_sweeps32(const float *W, int64_t n, double lam, const int32_t *pi,
                        const int32_t *pj, int64_t np, const double *inva, const double *g,
                        const double *aval, int nsweeps, double *D, float *U, Work &w,
                        bool chain64, cudaStream_t st, float *U2 = nullptr);

// ---- BCD-IC's Schur-complement line-search pieces (bcd.cu) ----
// Dl (n x n, zeroed by the caller) <- Delta from its pairs; *bad = 1 for a
// nonzero pair outside the block's rows and columns, 2 for an index outside [0, n).
cudaError_t bcd_scatter(const int32_t *pi, const int32_t *pj, const double *D, int64_t np, int64_t n,
                        const uint8_t *inI, double *Dl, int *bad, cudaStream_t st);
// out (m x m) = A[idx, idx]
cudaError_t bcd_gather(const double *A, int64_t n, const int32_t *idx, int64_t m, double *out, cudaStream_t st);
// Y = A_22^{-1} A_21, Z = A_22^{-1} Delta_21 (column c at offset c m2) from Ainv = A_22^{-1}
cudaError_t bcd_solve(const double *Ainv, int64_t m2, const double *A, const double *Dl, int64_t n,
                      const int32_t *idx1, int64_t m1, const int32_t *idx2, double *Y, double *Z, cudaStream_t st);
// M = B_0 + alpha B_1 + alpha^2 B_2 (m1 x m1)
cudaError_t bcd_assemble(const double *A, const double *Dl, int64_t n, const int32_t *idx1, int64_t m1,
                         const int32_t *idx2, int64_t m2, const double *Y, const double *Z, double alpha,
                         double *M, cudaStream_t st);

// ---- the batched solver (fused.cu) ----
// One problem of a fused launch: S and A_out are n x n FP64 on the device,
// A0 (optional) too; n <= GLASSO_FUSED_MAX_N.
constexpr int FUSED_THREADS = GLASSO_FUSED_MAX_N;  // one thread per column of a row
// device time of a fused solve per step class, indexed like the profile
// classes: 0 factorisations of the iterate, 1 inverses, 2 free-set scans and
// hierarchy, 3 CD sweeps, 4 line searches
constexpr int FUSED_CLASSES = 5;
struct FusedProblem {
    const double *S;
    const double *A0;
    double *A_out;
    double lambda, tol;
    int n, max_cycles, one_level, pad;
};
struct FusedResult {
    int status, cycles, relaxations, ls_trials;
    double objective, rel_kkt, max_kkt, logdet;
    long long nnz, max_nnz, sweeps;
    double flops;               // algorithmic FP64 operations of the dense steps and the sweeps
    double cls_ns[FUSED_CLASSES];  // device time per step class (ns)
    unsigned long long t0, t1;  // device global timer (ns) at the solve's start and end
};
// Workspace bytes of one CTA slot for problems of size <= nmax.
size_t fused_slot_bytes(int nmax);
// One persistent launch of `grid` CTAs over the paths (int2 {first, end}: a
// run of problems, each after the first warm started from its predecessor);
// next: one device int (zeroed here); arena: grid * slot_bytes.
cudaError_t fused_paths(const FusedProblem *probs, FusedResult *res, const int2 *paths, int npaths,
                        int *next, char *arena, size_t slot_bytes, int nmax, int grid,
                        cudaStream_t st);

}  // namespace glx
