// Host side of the library: the C ABI of include/glasso.h, device workspace,
// the ML-cycle driver (Algorithm 1 with nu = nu_c = 1 and the hierarchy of
// Section 7, relaxation = dense proximal Newton of Sections 5.1-5.2), the
// batch entry point and the asynchronous serving queue.
//
// Control flow per relaxation (device work on one stream, host reads a few
// scalars at the marked points):
//   W = A^{-1} from the current Cholesky factor            (dense.cu)
//   free set on C_l (+ KKT at level 0)          [sync]     (scan.cu)
//   per-pair data, U = 0, Delta = 0, CD sweeps             (scan.cu, cd.cu)
//   delta, tr(S Delta)                          [sync]     (scan.cu)
//   line search: T = A + alpha Delta, Cholesky  [sync per trial]
//   accept: A += alpha Delta, the trial's factor becomes the new factor.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "glasso_internal.h"

using namespace glx;

namespace glx {
std::atomic<long long> g_launches{0};
std::atomic<long long> g_paths[GLASSO_PATHS];
}

namespace {

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return fail_cuda(err, e_, #call);   \
    } while (0)

glasso_status fail_cuda(std::string &err, cudaError_t e, const char *what) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return GLASSO_ECUDA;
}

// GLASSO_TRACE=1 prints one line per relaxation to stderr (level, free pairs,
// objective, line-search regime and step, refinement steps).
bool trace_on() {
    static const bool on = [] {
        const char *e = getenv("GLASSO_TRACE");
        return e && *e && *e != '0';
    }();
    return on;
}

size_t footprint(int64_t n, int64_t m, int xbytes, bool screen = false) {
    const size_t nn = (size_t)n * (size_t)n;
    const size_t pairs = (size_t)n * (size_t)(n + 1) / 2;
    size_t b = 6 * nn * sizeof(double);                           // S A L T W U
    b += pairs * (6 * sizeof(int32_t) + 7 * sizeof(double) + 3);  // pair lists
    b += (size_t)n * ((n + 31) / 32) * sizeof(uint32_t);          // masks
    b += (size_t)(n + 1) * sizeof(long long) + (size_t)n * 6 * sizeof(double);
    if (m > 0) b += (size_t)m * n * (sizeof(double) + xbytes) + (size_t)n * sizeof(double);
    b += nn * (sizeof(int32_t) + sizeof(double));  // CSR of A (mixed precision)
    b += nn * sizeof(double);                      // CD interaction matrices (at most)
    b += (size_t)4 * n * ((n + 31) / 32 * 32) * sizeof(float);  // tensor-core factorisation planes
    if (screen) b += 4 * nn * sizeof(double) + (size_t)n * (4 * sizeof(int32_t) + sizeof(double));
    return b + (4u << 20);
}

template <typename T>
cudaError_t dalloc(T *&p, size_t count, cudaStream_t st) {
    if (p) {
        cudaError_t e = cudaFreeAsync(p, st);
        p = nullptr;
        if (e != cudaSuccess) return e;
    }
    if (count == 0) count = 1;
    return cudaMallocAsync((void **)&p, count * sizeof(T), st);
}

template <typename T>
void dfree(T *&p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
}

// The factorisation's side stream (lowest priority, so the serial path keeps
// the SMs it needs) and its two events, created on first use.
cudaError_t ensure_side(Work &w) {
    if (w.side) return cudaSuccess;
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e != cudaSuccess) return e;
    e = cudaStreamCreateWithPriority(&w.side, cudaStreamNonBlocking, lo);
    if (e != cudaSuccess) return e;
    e = cudaEventCreateWithFlags(&w.ev_a, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.ev_b, cudaEventDisableTiming);
    return e;
}

void work_free(Work &w, cudaStream_t st) {
    dfree(w.S, st); dfree(w.A, st); dfree(w.L, st); dfree(w.T, st); dfree(w.W, st); dfree(w.U, st);
    dfree(w.Xin, st); dfree(w.Xraw, st);
    dfree(w.fi, st); dfree(w.fj, st); dfree(w.fabsg, st); dfree(w.ftag, st); dfree(w.fsupp, st);
    dfree(w.pi, st); dfree(w.pj, st); dfree(w.pabsg, st); dfree(w.D, st);
    dfree(w.p_inva, st); dfree(w.p_g, st); dfree(w.p_a, st); dfree(w.p_s, st);
    dfree(w.mask, st); dfree(w.rowcnt, st); dfree(w.rowred, st); dfree(w.flags, st);
    dfree(w.blkcnt, st); dfree(w.redbuf, st);
    dfree(w.cd_part, st); dfree(w.xd, st); dfree(w.ldiag, st); dfree(w.sc, st);
    dfree(w.cd_k, st);
    dfree(w.fa, st);
    w.cap_cd_k = 0;
    dfree(w.csr_ptr, st); dfree(w.csr_col, st); dfree(w.csr_val, st); dfree(w.part, st);
    dfree(w.Wp, st); dfree(w.Qp, st); dfree(w.U2p, st); dfree(w.U3p, st); dfree(w.Xt, st);
    w.cap_mixed = w.cap_part = w.cap_xt = 0;
    dfree(w.scr_S, st); dfree(w.scr_A, st); dfree(w.scr_W, st); dfree(w.scr_A0, st);
    dfree(w.scr_diag, st); dfree(w.cc_parent, st); dfree(w.cc_size, st); dfree(w.cc_comp, st);
    dfree(w.scr_idx, st);
    w.cap_scr = w.cap_cc = 0;
    if (w.pcd_vec) cudaFreeAsync(w.pcd_vec, st);
    if (w.pcd_rows) cudaFreeAsync(w.pcd_rows, st);
    w.pcd_vec = nullptr;
    w.pcd_rows = nullptr;
    w.pcd_cap_np = w.pcd_cap_n = 0;
    if (w.sc_host) cudaFreeHost(w.sc_host);
    w.sc_host = nullptr;
    if (w.ev_a) cudaEventDestroy(w.ev_a);
    if (w.ev_b) cudaEventDestroy(w.ev_b);
    if (w.side) cudaStreamDestroy(w.side);
    w.ev_a = w.ev_b = nullptr;
    w.side = nullptr;
    w.cap_n = w.cap_pairs = w.cap_x = w.cap_xraw = w.cap_blk = w.cap_red = 0;
}

glasso_status work_ensure(Work &w, int64_t n, cudaStream_t st, std::string &err) {
    if (!w.sc) {
        CK(dalloc(w.sc, 1, st));
        CK(cudaMemsetAsync(w.sc, 0, sizeof(DevScalars), st));
        CK(cudaMallocHost((void **)&w.sc_host, sizeof(DevScalars)));
        CK(dalloc(w.redbuf, 3 * 1024, st));
        w.cap_red = 3 * 1024;
        CK(dalloc(w.cd_part, (size_t)2 * CD_MAX_CHUNKS * CD_B + (size_t)CD_B * CD_B, st));
        CK(dalloc(w.xd, 2 * NB * NB, st));
    }
    if (n <= w.cap_n) return GLASSO_OK;
    const size_t nn = (size_t)n * (size_t)n;
    const int64_t pairs = n * (n + 1) / 2;
    CK(dalloc(w.S, nn, st)); CK(dalloc(w.A, nn, st)); CK(dalloc(w.L, nn, st));
    CK(dalloc(w.T, nn, st)); CK(dalloc(w.W, nn, st)); CK(dalloc(w.U, nn, st));
    CK(dalloc(w.fi, pairs, st)); CK(dalloc(w.fj, pairs, st)); CK(dalloc(w.fabsg, pairs, st));
    CK(dalloc(w.ftag, pairs, st)); CK(dalloc(w.fsupp, pairs, st));
    CK(dalloc(w.pi, pairs, st)); CK(dalloc(w.pj, pairs, st)); CK(dalloc(w.pabsg, pairs, st));
    CK(dalloc(w.D, pairs, st));
    CK(dalloc(w.p_inva, pairs, st)); CK(dalloc(w.p_g, pairs, st)); CK(dalloc(w.p_a, pairs, st));
    CK(dalloc(w.p_s, pairs, st));
    CK(dalloc(w.flags, pairs, st));
    w.cap_blk = (pairs + 1023) / 1024 + 1;
    CK(dalloc(w.blkcnt, w.cap_blk, st));
    CK(dalloc(w.mask, (size_t)n * ((n + 31) / 32), st));
    CK(dalloc(w.rowcnt, n + 1, st));
    CK(dalloc(w.rowred, std::max((size_t)n * 6, (size_t)5 * 152), st));  // per-row stats / scan partials
    CK(dalloc(w.ldiag, n, st));
    w.cap_n = n;
    w.cap_pairs = pairs;
    return GLASSO_OK;
}

// Screening buffers: full-size copies of S, A, W and A0 (the sub-problem
// occupies S .. U), the component labels and the sub-problem's vertex list.
glasso_status work_ensure_labels(Work &w, int64_t n, cudaStream_t st, std::string &err) {
    if (n <= w.cap_cc) return GLASSO_OK;
    CK(dalloc(w.scr_diag, n, st));
    CK(dalloc(w.cc_parent, n, st)); CK(dalloc(w.cc_size, n, st));
    CK(dalloc(w.cc_comp, n, st)); CK(dalloc(w.scr_idx, n, st));
    w.cap_cc = n;
    return GLASSO_OK;
}

glasso_status work_ensure_screen(Work &w, int64_t n, cudaStream_t st, std::string &err) {
    glasso_status s = work_ensure_labels(w, n, st, err);
    if (s != GLASSO_OK || n <= w.cap_scr) return s;
    const size_t nn = (size_t)n * (size_t)n;
    CK(dalloc(w.scr_S, nn, st)); CK(dalloc(w.scr_A, nn, st));
    CK(dalloc(w.scr_W, nn, st)); CK(dalloc(w.scr_A0, nn, st));
    w.cap_scr = n;
    return GLASSO_OK;
}

glasso_status work_ensure_mixed(Work &w, int64_t n, cudaStream_t st, std::string &err) {
    if (n <= w.cap_mixed) return GLASSO_OK;
    const int64_t nt = (n + 31) / 32;
    const int64_t np2 = tc_pad(n) * tc_pad(n);
    CK(dalloc(w.csr_ptr, n + 1, st));
    CK(dalloc(w.csr_col, (size_t)n * n + n, st));
    CK(dalloc(w.csr_val, (size_t)n * n + n, st));
    w.cap_part = nt * nt + 1024;
    CK(dalloc(w.part, w.cap_part, st));
    CK(dalloc(w.Wp, np2, st));
    CK(dalloc(w.Qp, np2, st));
    CK(dalloc(w.U2p, np2, st));
    CK(dalloc(w.U3p, np2, st));
    CK(dalloc(w.fa, (size_t)4 * n * tc_pad(n), st));
    w.cap_mixed = n;
    return GLASSO_OK;
}

glasso_status work_ensure_x(Work &w, int64_t m, int64_t n, int xbytes, cudaStream_t st,
                            std::string &err) {
    const int64_t need = m * n + n;
    if (need > w.cap_x) {
        CK(dalloc(w.Xin, need, st));
        w.cap_x = need;
    }
    const int64_t rawb = m * n * xbytes;
    if (rawb > w.cap_xraw) {
        CK(dalloc(w.Xraw, rawb, st));
        w.cap_xraw = rawb;
    }
    return GLASSO_OK;
}

// ---- validation -----------------------------------------------------------
__global__ void k_check_sym(const double *__restrict__ S, int64_t n, int *bad_sym, int *bad_nan,
                            double *maxabs_part) {
    __shared__ double red[256];
    double mx = 0.0;
    int nan = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        double v = S[t];
        if (!isfinite(v)) nan = 1;
        mx = fmax(mx, fabs(v));
    }
    if (nan) atomicExch(bad_nan, 1);
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) maxabs_part[blockIdx.x] = red[0];
}

__global__ void k_check_sym2(const double *__restrict__ S, int64_t n, const double *maxabs_part,
                             int nparts, int *bad_sym) {
    __shared__ double mx;
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int p = 0; p < nparts; ++p) m = fmax(m, maxabs_part[p]);
        mx = m;
    }
    __syncthreads();
    const double tol = 1e-12 * mx;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = t / n, j = t % n;
        if (j > i && fabs(S[t] - S[j * n + i]) > tol) atomicExch(bad_sym, 1);
    }
}

// Returns OK, or EINVAL on NaN/Inf or asymmetry beyond 1e-12 max|S|.
glasso_status check_symmetric(Work &w, const double *M, int64_t n, cudaStream_t st,
                              std::string &err) {
    CK(cudaMemsetAsync(w.sc, 0, sizeof(DevScalars), st));
    int *bad_nan = &w.sc->err;
    int *bad_sym = &w.sc->bad_sym;
    const int parts = 256;
    k_check_sym<<<parts, 256, 0, st>>>(M, n, bad_sym, bad_nan, w.redbuf);
    counted(1);
    k_check_sym2<<<parts, 256, 0, st>>>(M, n, w.redbuf, parts, bad_sym);
    counted(1);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(w.sc_host, w.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (w.sc_host->err || w.sc_host->bad_sym) return GLASSO_EINVAL;
    return GLASSO_OK;
}

// ---- the solver -------------------------------------------------------------
struct Prof {
    bool on = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
    double ms[GLASSO_PROF_CLASSES] = {0};  // indexes as in glasso.h
    long long count[GLASSO_PROF_CLASSES] = {0};
    double work[GLASSO_PROF_CLASSES] = {0};
    std::vector<double> pend_work;
    long long kernels_base = 0;
    long long paths_base[GLASSO_PATHS] = {0};
};

struct Solver {
    Work &w;
    cudaStream_t st;
    std::string &err;
    Prof *prof;
    int precision = GLASSO_FP64;
    int inner = GLASSO_INNER_CD;  // Newton-direction solver of the relaxations
    glasso_status sync() {
        CK(cudaMemcpyAsync(w.sc_host, w.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return GLASSO_OK;
    }
    void mark_begin(int cls, cudaEvent_t &b) {
        if (!prof || !prof->on) return;
        cudaEventCreate(&b);
        cudaEventRecord(b, st);
        (void)cls;
    }
    void mark_end(int cls, cudaEvent_t b, double work) {
        if (!prof || !prof->on) return;
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, st);
        prof->ev.push_back({cls, {b, e}});
        prof->pend_work.push_back(work);
    }
};

void prof_collect(Prof *prof) {
    if (!prof) return;
    for (size_t k = 0; k < prof->ev.size(); ++k) {
        float ms = 0.f;
        cudaEventSynchronize(prof->ev[k].second.second);
        cudaEventElapsedTime(&ms, prof->ev[k].second.first, prof->ev[k].second.second);
        int c = prof->ev[k].first;
        prof->ms[c] += ms;
        prof->count[c] += 1;
        prof->work[c] += prof->pend_work[k];
        cudaEventDestroy(prof->ev[k].second.first);
        cudaEventDestroy(prof->ev[k].second.second);
    }
    prof->ev.clear();
    prof->pend_work.clear();
}

// PCD-CG as the inner solver: Section 8's relative precision, and an
// iteration cap that the precision normally reaches long before.
constexpr int kPcdIters = 500;

// The inner solver of one relaxation: GLASSO_INNER_AUTO takes PCD-CG when
// the CD sweeps' serial chain would be long (pairs x sweeps coordinate
// updates, each a dependent step of the chain) and CD sweeps otherwise,
// where PCD-CG's fixed cost (the pair CSR and a persistent launch with grid
// barriers) would dominate.
int64_t auto_pcd_work() {
    static const int64_t v = [] {
        const char *ev = getenv("GLASSO_AUTO_PCD_WORK");
        const long long x = ev ? atoll(ev) : 0;
        return (int64_t)(x > 0 ? x : GLASSO_AUTO_PCD_WORK);
    }();
    return v;
}
bool pick_pcd(int inner, int64_t np, int nsweeps) {
    if (inner == GLASSO_INNER_PCD_CG) return true;
    return inner == GLASSO_INNER_AUTO && np * (int64_t)nsweeps >= auto_pcd_work();
}
constexpr double kPcdRtol = 1e-4;
// Algorithmic bytes of one PCD-CG iteration with word size ws: the SpMM reads
// the 2 np rows of W its pairs name and writes V^T (n^2), the SDDMM reads two
// rows per pair.
double pcd_bytes(int64_t np, double nd, double ws) { return (4.0 * (double)np * nd + nd * nd) * ws; }

// Sums a caller combining several solves needs beyond glasso_info.
struct CoreSums {
    double l1 = 0.0;  // ||A||_1 at return
};

// The continuation's stage values (end of Section 2; the schedule of
// Section 8): lambda_4 halfway between lambda and lambda_max = max_{i != j}
// |S_ij| (the smallest lambda whose minimiser is diagonal; at most 1 on the
// paper's normalised data, where it takes lambda_4 = (1 + lambda) / 2), then
// lambda_3, lambda_2 evenly spaced down to lambda.  Returns the stage count:
// 3, or 0 when lambda_max <= lambda.
int continuation_lambdas(unsigned long long smax_bits, double lam, double out[3]) {
    double lmax;
    memcpy(&lmax, &smax_bits, sizeof(lmax));
    if (!(lmax > lam)) return 0;
    const double l4 = 0.5 * (lmax + lam);
    for (int s = 4; s >= 2; --s) out[4 - s] = lam + (double)(s - 1) * (l4 - lam) / 3.0;
    return 3;
}

// Runs the ML-cycle solve on w.S (and w.A if have_A0).  Leaves the iterate in
// w.A and its inverse in w.W when W is requested (want_W).
glasso_status solve_core(Solver &sv, int64_t n, double lam, double tol, int max_cycles,
                         bool have_A0, bool want_W, bool one_level, bool continuation,
                         glasso_info *info, CoreSums *sums = nullptr) {
    Work &w = sv.w;
    cudaStream_t st = sv.st;
    std::string &err = sv.err;
    DevScalars *sc = w.sc;
    DevScalars *h = w.sc_host;
    const double sigma = 1e-4;
    const int max_trials = 30;
    const double nd = (double)n;
    const double flop_chol = nd * nd * nd / 3.0, flop_inv = 2.0 * nd * nd * nd / 3.0;
    int cycles = 0, relax = 0, lstrials = 0;
    long long inner_iters = 0;
    double F = 0.0, logdet = 0.0, trSA = 0.0, l1 = 0.0, relkkt = INFINITY, maxkkt = INFINITY;
    long long nnz = 0, max_nnz = 0;
    glasso_status status = GLASSO_EMAXITER;
    bool W_valid = false, fresh_scan = false;
    int64_t nf = 0;
    cudaEvent_t eb;

    CK(cudaMemsetAsync(sc, 0, sizeof(DevScalars), st));
    if (!have_A0) CK(init_diag(w.S, n, lam, w.A, sc, st));
    CK(cudaMemcpyAsync(w.L, w.A, (size_t)(n * n) * sizeof(double), cudaMemcpyDeviceToDevice, st));
    sv.mark_begin(0, eb);
    CK(potrf(w.L, n, w.xd, w.ldiag, sc, st));
    sv.mark_end(0, eb, flop_chol);
    if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
    if (h->err || h->info != 0) return GLASSO_ENOTPD;
    logdet = h->logdet;
    sv.mark_begin(1, eb);
    CK(inverse(w.L, n, w.W, w.T, w.U, st));
    sv.mark_end(1, eb, flop_inv);
    W_valid = true;
    if (continuation) CK(offdiag_absmax(w.S, n, sc, st));
    // initial free set (Section 7 footnote): {|S_ij| > lambda} united with supp(A0)
    CK(scan_full(w.S, w.W, w.A, n, lam, 1, w, w.fi, w.fj, w.fabsg, sc, st));
    if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
    nf = h->count;
    trSA = h->trSA;
    l1 = h->l1;
    F = -logdet + trSA + lam * l1;

    double stage_lam[3];
    const int nstage = continuation ? continuation_lambdas(h->smax_bits, lam, stage_lam) : 0;
    double lam_F = lam;  // the lambda that F currently includes
    // k < 0: the continuation stages, one level-0 relaxation each at lambda_s
    for (int k = -nstage; k < max_cycles; ++k) {
        const double lk = k < 0 ? stage_lam[k + nstage] : lam;
        if (k >= 0) cycles = k + 1;
        const int nsweeps = k < 0 ? 1 : std::min(1 + k / 3, 10);
        if (lk != lam_F) {
            F = -logdet + trSA + lk * l1;
            lam_F = lk;
        }
        // the one-level method (Section 8's comparison) and the continuation
        // stages: the full free set, no hierarchy
        int Lv = 0;
        if (!one_level && k >= 0) {
            CK(support_flags(w.A, n, w.fi, w.fj, nf, w.fsupp, st));
            CK(hierarchy(w.fabsg, w.fsupp, nf, w.ftag, sc, st));
            if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
            Lv = h->levels;
        }
        for (int l = Lv; l >= 0; --l) {
            fresh_scan = false;
            if (!W_valid) {
                sv.mark_begin(1, eb);
                CK(inverse(w.L, n, w.W, w.T, w.U, st));
                sv.mark_end(1, eb, flop_inv);
                W_valid = true;
            }
            int64_t np;
            if (l == 0) {
                sv.mark_begin(2, eb);
                CK(scan_full(w.S, w.W, w.A, n, lk, 0, w, w.pi, w.pj, w.pabsg, sc, st));
                sv.mark_end(2, eb, 3.0 * nd * (nd + 1) / 2 * 8.0);
                if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
                np = h->count;
                trSA = h->trSA;
                l1 = h->l1;
                nnz = h->nnz;
                max_nnz = std::max(max_nnz, nnz);
                F = -logdet + trSA + lk * l1;
                relkkt = h->kkt_sum / l1;
                maxkkt = h->kkt_max;
                fresh_scan = k >= 0;  // a stage scan is at lambda_s, not lambda
                CK(cudaMemcpyAsync(w.fi, w.pi, np * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(w.fj, w.pj, np * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(w.fabsg, w.pabsg, np * sizeof(double), cudaMemcpyDeviceToDevice, st));
                nf = np;
                if (k >= 0 && relkkt <= tol) {
                    status = GLASSO_OK;
                    goto done;
                }
            } else {
                CK(scan_cand(w.S, w.W, w.A, n, lk, w.fi, w.fj, w.ftag, l, nf, w, w.pi, w.pj,
                             nullptr, sc, st));
                if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
                np = h->count;
            }
            ++relax;
            if (np == 0) continue;
            CK(pair_prep(w.S, w.W, w.A, n, lk, w.pi, w.pj, np, w.p_inva, w.p_g, w.p_a, w.p_s, st));
            CK(cudaMemsetAsync(w.U, 0, (size_t)(n * n) * sizeof(double), st));
            CK(cudaMemsetAsync(w.D, 0, np * sizeof(double), st));
            sv.mark_begin(3, eb);
            if (pick_pcd(sv.inner, np, nsweeps)) {
                // PCD-CG to relative precision 1e-4 (Section 8); T is free until the line search
                int its = 0;
                const cudaError_t pe = pcd(w.W, n, lk, w.pi, w.pj, np, w.p_inva, w.p_g, w.p_a, kPcdIters, 1,
                                           kPcdRtol, w.D, w.U, w.T, false, w, st, &its);
                if (pe == cudaErrorLaunchTimeout) {
                    err = "PCD-CG: a bounded grid-barrier wait expired";
                    return GLASSO_ETIMEOUT;
                }
                CK(pe);
                inner_iters += its;
                sv.mark_end(3, eb, (double)its * pcd_bytes(np, nd, 8.0));
            } else {
                CK(cd_sweeps(w.W, n, lk, w.pi, w.pj, np, w.p_inva, w.p_g, w.p_a, nsweeps, w.D, w.U, w, st));
                inner_iters += nsweeps;
                sv.mark_end(3, eb, (double)nsweeps * (double)np * 6.0 * nd * 8.0);
            }
            CK(ls_delta(w.p_g, w.p_a, w.p_s, w.D, w.pi, w.pj, np, lk, w, sc, st));
            if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
            if (h->bar_err) {
                err = "CD sweep: a bounded grid-barrier wait expired";
                return GLASSO_ETIMEOUT;
            }
            if (!h->moved) continue;
            {
                const double delta = h->delta, trSD = h->trSD;
                const double epsF = 1e-12 * std::max(fabs(F), nd);
                double alpha = 1.0;
                bool ok = false;
                double FT = 0.0, dl1 = 0.0, ldT = 0.0;
                for (int t = 0; t < max_trials; ++t) {
                    CK(ls_build_trial(w.A, w.T, n, w.pi, w.pj, w.p_a, w.D, np, alpha, st));
                    sv.mark_begin(4, eb);
                    CK(potrf(w.T, n, w.xd, w.ldiag, sc, st));
                    sv.mark_end(4, eb, flop_chol);
                    CK(ls_dl1(w.p_a, w.D, w.pi, w.pj, np, alpha, w, sc, st));
                    if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
                    ++lstrials;
                    if (h->info == 0 && !w.dbg_ls_reject) {
                        ldT = h->logdet;
                        dl1 = h->dl1;
                        FT = -ldT + trSA + alpha * trSD + lk * (l1 + dl1);
                        if (FT <= F + sigma * alpha * delta + epsF) {
                            ok = true;
                            break;
                        }
                    }
                    alpha *= 0.5;
                }
                if (!ok) {
                    status = GLASSO_ELINESEARCH;
                    goto done;
                }
                CK(ls_apply(w.A, n, w.pi, w.pj, w.p_a, w.D, np, alpha, st));
                if (trace_on())
                    fprintf(stderr, "glasso[fp64] cycle %d level %d pairs %lld F %.15g dF %.3e alpha %g trials %d "
                            "inner %lld relkkt %.3e\n",
                            k, l, (long long)np, FT, FT - F, alpha, lstrials, inner_iters, relkkt);
                std::swap(w.L, w.T);
                logdet = ldT;
                trSA += alpha * trSD;
                l1 += dl1;
                F = FT;
                W_valid = false;
            }
        }
    }
done:
    if (!fresh_scan) {
        if (!W_valid) {
            CK(inverse(w.L, n, w.W, w.T, w.U, st));
            W_valid = true;
        }
        CK(scan_full(w.S, w.W, w.A, n, lam, 0, w, w.pi, w.pj, w.pabsg, sc, st));
        if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
        trSA = h->trSA;
        l1 = h->l1;
        nnz = h->nnz;
        F = -logdet + trSA + lam * l1;
        relkkt = h->kkt_sum / l1;
        maxkkt = h->kkt_max;
    }
    max_nnz = std::max(max_nnz, nnz);
    (void)want_W;
    if (sums) sums->l1 = l1;
    if (info) {
        info->status = status;
        info->cycles = cycles;
        info->relaxations = relax;
        info->ls_trials = lstrials;
        info->objective = F;
        info->rel_kkt = relkkt;
        info->max_kkt = maxkkt;
        info->logdet = logdet;
        info->nnz = nnz;
        info->max_nnz = max_nnz;
        info->inner_iters = inner_iters;
    }
    return status;
}

// ---------------------------------------------------------------------------
// Mixed-precision solve (GLASSO_MIXED).  Same ML-cycle and relaxation as
// solve_core; the differences are confined to how W and the line-search
// log-det are obtained (mixed.cu):
//  * W (FP64) comes from the previous W by Newton-Schulz refinement against
//    the new A (TF32 GEMM corrections, residual and sum in double-float FP32
//    arithmetic), or after a large step from an FP32 Cholesky + inverse, then
//    refined the same way;
//  * the CD sweep runs on FP32 copies of W and U (an inexact Hessian, which
//    the convergence theory of Section 4.1 allows), with the FP64 gradient;
//  * the line search uses the log-det series when its remainder bound is below
//    the objective's FP64 resolution (positive definiteness then holds by
//    construction, and the increment is exact enough to track log det A), and
//    otherwise an FP32 Cholesky (FP64 diagonal blocks and log accumulation)
//    whose log-det error is taken as n 2^-20.
glasso_status solve_core_mixed(Solver &sv, int64_t n, double lam, double tol, int max_cycles,
                               bool have_A0, bool one_level, bool continuation, glasso_info *info,
                               CoreSums *sums = nullptr) {
    Work &w = sv.w;
    cudaStream_t st = sv.st;
    std::string &err = sv.err;
    DevScalars *sc = w.sc;
    DevScalars *h = w.sc_host;
    {
        glasso_status s0 = work_ensure_mixed(w, n, st, err);
        if (s0 != GLASSO_OK) return s0;
    }
    const size_t nn = (size_t)n * (size_t)n;
    const int64_t ldf = tc_pad(n);
    float *FA = w.fa, *FX = FA + n * ldf, *FXt = FX + n * ldf, *FZ = FXt + n * ldf;
    // W during refinement: W32 + Wlo (double-float); W32 is also the FP32 copy
    // the sweep and the series read, W64 the FP64 W after refinement
    float *W32 = (float *)w.L, *R32 = W32 + nn;
    float *U32 = (float *)w.U, *Wlo = U32 + nn;
    double *W64 = w.W;
    const double sigma = 1e-4;
    const int max_trials = 30;
    const double nd = (double)n;
    const double e_chol = nd * 0x1p-20;  // FP32 Cholesky log-det error allowance
    const double ns_tol = 1e-11;
    const int max_ns = 8;
    int cycles = 0, relax = 0, lstrials = 0;
    long long inner_iters = 0;
    double F = 0.0, logdet = 0.0, trSA = 0.0, l1 = 0.0, relkkt = INFINITY, maxkkt = INFINITY;
    long long nnz = 0, max_nnz = 0;
    glasso_status status = GLASSO_EMAXITER;
    bool W_valid = false, fresh_scan = false, last_chol = false;
    int64_t nf = 0;
    cudaEvent_t eb;

    // W = X^T X from the inverse factor X = L^{-1} of the last tensor-core
    // factorisation (FXt = X^T), then refined.
    auto factor_inverse = [&]() -> glasso_status {
        sv.mark_begin(1, eb);
        CK(lauum_tc(FXt, n, ldf, W32, n, sc, st));
        CK(to_f64(W32, W64, (int64_t)nn, st));
        CK(cudaMemsetAsync(Wlo, 0, nn * sizeof(float), st));
        sv.mark_end(1, eb, nd * nd * nd / 3.0);
        return GLASSO_OK;
    };
    auto factor_wait = [&]() -> glasso_status {
        if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
        if (h->tc_err) {
            err = "tensor-core factorisation: a bounded wait expired (code " + std::to_string(h->tc_err) + ")";
            return GLASSO_ETIMEOUT;
        }
        return GLASSO_OK;
    };
    auto fresh_factor = [&]() -> glasso_status {
        CK(trial32(w.A, FA, n, ldf, w.pi, w.pj, w.p_a, w.D, 0, 0.0, st));
        CK(ensure_side(w));
        CK(cholinv_tc(FA, n, ldf, FX, FXt, FZ, w.ldiag, sc, st, w.side, w.ev_a, w.ev_b, w.dbg_dag_tiles, w.dag_share));
        glasso_status s2 = factor_wait();
        if (s2 != GLASSO_OK) return s2;
        if (h->info != 0) return GLASSO_ENOTPD;
        return factor_inverse();
    };
    int ns_steps = 0;
    auto refine = [&]() -> glasso_status {
        CK(build_csr(w.A, n, w.csr_ptr, w.csr_col, w.csr_val, st));
        bool restarted = false;
        ns_steps = 0;
        // hi alternates between W32 and a second buffer (the GEMM reads the
        // current one while its epilogue writes the next)
        float *hcur = W32, *hnext = reinterpret_cast<float *>(w.T) + nn;
        for (int it = 0; it < max_ns; ++it, ++ns_steps) {
            CK(residual(w.csr_ptr, w.csr_col, w.csr_val, hcur, Wlo, n, R32, w.rowred, sc, st));
            if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
            if (h->tc_err) {
                err = "tensor-core GEMM: a bounded wait expired (code " + std::to_string(h->tc_err) + ")";
                return GLASSO_ETIMEOUT;
            }
            if (h->ns_max <= ns_tol) break;
            if (!(sqrt(h->ns_fro2) < 0.9)) {
                if (restarted) break;
                restarted = true;
                glasso_status s2 = fresh_factor();
                if (s2 != GLASSO_OK) return s2;
                hcur = W32;  // the fresh factor's W
                hnext = reinterpret_cast<float *>(w.T) + nn;
                it = -1;
                continue;
            }
            sv.mark_begin(5, eb);
            CK(ns_gemm_tc(hcur, hnext, Wlo, R32, n, w.Wp, w.Qp, &sc->tc_err, st));
            path_hit(GLASSO_PATH_NS_STEPS);
            sv.mark_end(5, eb, nd * nd * nd);
            std::swap(hcur, hnext);
        }
        if (hcur != W32)
            CK(cudaMemcpyAsync(W32, hcur, nn * sizeof(float), cudaMemcpyDeviceToDevice, st));
        CK(join64(W32, Wlo, W64, (int64_t)nn, st));  // the FP64 W of the gradient and the pairs
        return GLASSO_OK;
    };
    auto update_W = [&]() -> glasso_status {
        if (last_chol) {
            glasso_status s2 = factor_inverse();
            if (s2 != GLASSO_OK) return s2;
        }
        return refine();
    };

    CK(cudaMemsetAsync(sc, 0, sizeof(DevScalars), st));
    if (!have_A0) {
        CK(init_diag(w.S, n, lam, w.A, sc, st));
        CK(diag_inverse(w.A, n, W64, w.ldiag, sc, st));
        CK(split64(W64, W32, Wlo, (int64_t)nn, st));
        if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
        if (h->err) return GLASSO_ENOTPD;
        logdet = h->logdet;
    } else {
        glasso_status s2 = fresh_factor();
        if (s2 != GLASSO_OK) return s2;
        logdet = h->logdet;
        s2 = refine();
        if (s2 != GLASSO_OK) return s2;
    }
    W_valid = true;
    if (continuation) CK(offdiag_absmax(w.S, n, sc, st));
    CK(scan_full(w.S, W64, w.A, n, lam, 1, w, w.fi, w.fj, w.fabsg, sc, st));
    if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
    nf = h->count;
    trSA = h->trSA;
    l1 = h->l1;
    F = -logdet + trSA + lam * l1;

    double stage_lam[3];
    const int nstage = continuation ? continuation_lambdas(h->smax_bits, lam, stage_lam) : 0;
    double lam_F = lam;  // the lambda that F currently includes
    // k < 0: the continuation stages, one level-0 relaxation each at lambda_s
    for (int k = -nstage; k < max_cycles; ++k) {
        const double lk = k < 0 ? stage_lam[k + nstage] : lam;
        if (k >= 0) cycles = k + 1;
        const int nsweeps = k < 0 ? 1 : std::min(1 + k / 3, 10);
        if (lk != lam_F) {
            F = -logdet + trSA + lk * l1;
            lam_F = lk;
        }
        // the one-level method (Section 8's comparison) and the continuation
        // stages: the full free set, no hierarchy
        int Lv = 0;
        if (!one_level && k >= 0) {
            CK(support_flags(w.A, n, w.fi, w.fj, nf, w.fsupp, st));
            CK(hierarchy(w.fabsg, w.fsupp, nf, w.ftag, sc, st));
            if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
            Lv = h->levels;
        }
        for (int l = Lv; l >= 0; --l) {
            fresh_scan = false;
            if (!W_valid) {
                glasso_status s2 = update_W();
                if (s2 != GLASSO_OK) return s2;
                W_valid = true;
            }
            int64_t np;
            if (l == 0) {
                sv.mark_begin(2, eb);
                CK(scan_full(w.S, W64, w.A, n, lk, 0, w, w.pi, w.pj, w.pabsg, sc, st));
                sv.mark_end(2, eb, 3.0 * nd * (nd + 1) / 2 * 8.0);
                if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
                np = h->count;
                trSA = h->trSA;
                l1 = h->l1;
                nnz = h->nnz;
                max_nnz = std::max(max_nnz, nnz);
                F = -logdet + trSA + lk * l1;
                relkkt = h->kkt_sum / l1;
                maxkkt = h->kkt_max;
                fresh_scan = k >= 0;  // a stage scan is at lambda_s, not lambda
                CK(cudaMemcpyAsync(w.fi, w.pi, np * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(w.fj, w.pj, np * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(w.fabsg, w.pabsg, np * sizeof(double), cudaMemcpyDeviceToDevice, st));
                nf = np;
                if (k >= 0 && relkkt <= tol) {
                    status = GLASSO_OK;
                    goto done;
                }
            } else {
                CK(scan_cand(w.S, W64, w.A, n, lk, w.fi, w.fj, w.ftag, l, nf, w, w.pi, w.pj,
                             nullptr, sc, st));
                if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
                np = h->count;
            }
            ++relax;
            if (np == 0) continue;
            CK(pair_prep(w.S, W64, w.A, n, lk, w.pi, w.pj, np, w.p_inva, w.p_g, w.p_a, w.p_s, st));
            CK(cudaMemsetAsync(U32, 0, nn * sizeof(float), st));
            CK(cudaMemsetAsync(w.D, 0, np * sizeof(double), st));
            sv.mark_begin(3, eb);
            // FP32 resolution chain while the iterate is far from the optimum; FP64
            // once the relative KKT residual is small, where the Newton step must be
            // resolved to the gradient's FP64 accuracy
            // (the FP64 buffer T is free in this path: it holds the second copy of U)
            if (pick_pcd(sv.inner, np, nsweeps)) {
                // PCD-CG with FP32 products (T's FP32 halves are free until the next refinement)
                int its = 0;
                const cudaError_t pe = pcd32(W32, n, lk, w.pi, w.pj, np, w.p_inva, w.p_g, w.p_a, kPcdIters, 1,
                                             kPcdRtol, w.D, U32, (float *)w.T, false, w, st, &its);
                if (pe == cudaErrorLaunchTimeout) {
                    err = "PCD-CG: a bounded grid-barrier wait expired";
                    return GLASSO_ETIMEOUT;
                }
                CK(pe);
                inner_iters += its;
                sv.mark_end(3, eb, (double)its * pcd_bytes(np, nd, 4.0));
            } else {
                CK(cd_sweeps32(W32, n, lk, w.pi, w.pj, np, w.p_inva, w.p_g, w.p_a, nsweeps, w.D, U32, w,
                               relkkt <= 1e-6, st, (float *)w.T));
                inner_iters += nsweeps;
                sv.mark_end(3, eb, (double)nsweeps * (double)np * 6.0 * nd * 4.0);
            }
            CK(ls_delta(w.p_g, w.p_a, w.p_s, w.D, w.pi, w.pj, np, lk, w, sc, st));
            CK(series_terms(W64, n, w.pi, w.pj, w.D, np, U32, w.part, w.cap_part, sc, st));
            if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
            if (h->bar_err) {
                err = "CD sweep: a bounded grid-barrier wait expired";
                return GLASSO_ETIMEOUT;
            }
            if (!h->moved) continue;
            {
                const double delta = h->delta, trSD = h->trSD;
                const double t1 = h->t1, t2 = std::max(h->t2, 0.0);
                const double epsF = 1e-12 * std::max(fabs(F), nd);
                // per-step budget of the tracked log-det (the stated objective accuracy)
                const double track = 1e-10 * std::max(fabs(F), nd);
                double t3 = 0.0, t4 = 0.0, t5 = 0.0, t6 = 0.0;
                bool high = false;
                double alpha = 1.0;
                bool ok = false, chol = false;
                double FT = 0.0, dl1 = 0.0, dld = 0.0;
                int nterms = 0;
                for (int t = 0; t < max_trials; ++t) {
                    const double rho = alpha * sqrt(t2);
                    CK(ls_dl1(w.p_a, w.D, w.pi, w.pj, np, alpha, w, sc, st));
                    double errb = INFINITY;
                    bool pd = true;
                    // log det(A + alpha Delta) - log det A = sum_k (-1)^{k+1} alpha^k t_k / k,
                    // remainder after K terms <= rho^{K+1} / ((K+1)(1 - rho)); rho < 1
                    // also proves A + alpha Delta positive definite
                    nterms = 0;
                    if (rho < 0.5) {
                        const double r2 = rho * rho * rho / (3.0 * (1.0 - rho)) + 1e-6 * alpha * alpha * t2;
                        if (r2 <= track) {
                            nterms = 2;
                            errb = r2;
                        } else {
                            if (!high) {
                                CK(series_high(U32, n, w.Wp, w.Qp, w.U2p, w.U3p, w.part, w.cap_part, sc, st));
                                if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
                                if (h->tc_err) {
                                    err = "tensor-core GEMM: a bounded wait expired";
                                    return GLASSO_ETIMEOUT;
                                }
                                t3 = h->t3; t4 = h->t4; t5 = h->t5; t6 = h->t6;
                                high = true;
                            }
                            const double r7 = pow(rho, 7.0) / (7.0 * (1.0 - rho));
                            // t3 .. t6 from split-TF32 products: relative error
                            // about (n / 8 + 2) 2^-24 of each term
                            const double eps_t = (nd / 8.0 + 2.0) * 0x1p-24;
                            const double terr = eps_t * (pow(rho, 3.0) / 3 + pow(rho, 4.0) / 4 +
                                                         pow(rho, 5.0) / 5 + pow(rho, 6.0) / 6);
                            if (r7 + terr + 1e-6 * alpha * alpha * t2 <= track) {
                                nterms = 6;
                                errb = r7 + terr + 1e-6 * alpha * alpha * t2;
                            }
                        }
                    }
                    if (nterms > 0) {
                        path_hit(nterms == 2 ? GLASSO_PATH_LS_SERIES2 : GLASSO_PATH_LS_SERIES6);
                        chol = false;
                        if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
                        const double a2 = alpha * alpha, a3 = a2 * alpha;
                        dld = alpha * t1 - 0.5 * a2 * t2;
                        if (nterms == 6)
                            dld += a3 * t3 / 3.0 - a2 * a2 * t4 / 4.0 + a3 * a2 * t5 / 5.0 - a3 * a3 * t6 / 6.0;
                    } else {
                        chol = true;
                        CK(trial32(w.A, FA, n, ldf, w.pi, w.pj, w.p_a, w.D, np, alpha, st));
                        sv.mark_begin(4, eb);
                        CK(ensure_side(w));
        CK(cholinv_tc(FA, n, ldf, FX, FXt, FZ, w.ldiag, sc, st, w.side, w.ev_a, w.ev_b, w.dbg_dag_tiles, w.dag_share));
                        sv.mark_end(4, eb, 2.0 * nd * nd * nd / 3.0);
                        glasso_status s2 = factor_wait();
                        if (s2 != GLASSO_OK) return s2;
                        pd = h->info == 0;
                        dld = h->logdet - logdet;
                        errb = 2.0 * e_chol;
                    }
                    ++lstrials;
                    if (pd && !w.dbg_ls_reject) {
                        dl1 = h->dl1;
                        FT = F - dld + alpha * trSD + lk * dl1;
                        if (FT <= F + sigma * alpha * delta + errb + epsF) {
                            ok = true;
                            break;
                        }
                    }
                    alpha *= 0.5;
                }
                if (!ok) {
                    status = GLASSO_ELINESEARCH;
                    goto done;
                }
                CK(ls_apply(w.A, n, w.pi, w.pj, w.p_a, w.D, np, alpha, st));
                if (trace_on())
                    fprintf(stderr,
                            "glasso[mixed] cycle %d level %d pairs %lld F %.12g dF %.3e rho %.3e "
                            "alpha %g regime %s terms %d ns_prev %d relkkt %.3e\n",
                            k, l, (long long)np, FT, FT - F, alpha * sqrt(t2), alpha,
                            chol ? "chol32" : "series", nterms, ns_steps, relkkt);
                logdet += dld;
                trSA += alpha * trSD;
                l1 += dl1;
                F = FT;
                W_valid = false;
                last_chol = chol;
            }
        }
    }
done:
    if (!fresh_scan) {
        if (!W_valid) {
            glasso_status s2 = update_W();
            if (s2 != GLASSO_OK) return s2;
            W_valid = true;
        }
        CK(scan_full(w.S, W64, w.A, n, lam, 0, w, w.pi, w.pj, w.pabsg, sc, st));
        if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
        trSA = h->trSA;
        l1 = h->l1;
        nnz = h->nnz;
        F = -logdet + trSA + lam * l1;
        relkkt = h->kkt_sum / l1;
        maxkkt = h->kkt_max;
    }
    max_nnz = std::max(max_nnz, nnz);
    if (sums) sums->l1 = l1;
    if (info) {
        info->status = status;
        info->cycles = cycles;
        info->relaxations = relax;
        info->ls_trials = lstrials;
        info->objective = F;
        info->rel_kkt = relkkt;
        info->max_kkt = maxkkt;
        info->logdet = logdet;
        info->nnz = nnz;
        info->max_nnz = max_nnz;
        info->inner_iters = inner_iters;
    }
    return status;
}

bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

// Stage the problem's S (or X -> S) and A0 on the device in w.
glasso_status form_S_ctx(Work &w, cudaStream_t st, int precision, const void *X, int dtype,
                         int64_t m, int64_t n, int center, double *S, std::string &err) {
    if (precision == GLASSO_MIXED && dtype == GLASSO_F32) {
        // TF32 tensor cores with FP32 accumulation (the FP32-sample workload)
        const int64_t need = n * tc_pad(m);
        if (need > w.cap_xt) {
            CK(dalloc(w.Xt, need, st));
            w.cap_xt = need;
        }
        double *mu = nullptr;
        if (center) {
            mu = w.Xin + m * n;  // n doubles of the staging buffer
            CK(form_S(X, dtype, m, n, 2, S, w.Xin, st));  // mode 2: column means only
        }
        CK(cudaMemsetAsync(&w.sc->tc_err, 0, sizeof(int), st));
        CK(syrk_tc(X, dtype, m, n, mu, S, w.Xt, &w.sc->tc_err, st));
        CK(cudaMemcpyAsync(w.sc_host, w.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (w.sc_host->tc_err) {
            err = "tensor-core GEMM: a bounded wait expired (code " + std::to_string(w.sc_host->tc_err) + ")";
            return GLASSO_ETIMEOUT;
        }
        return GLASSO_OK;
    }
    CK(form_S(X, dtype, m, n, center, S, w.Xin, st));
    return GLASSO_OK;
}

glasso_status stage_problem(Work &w, cudaStream_t st, const glasso_problem *p, std::string &err,
                            int precision) {
    const int64_t n = p->n;
    const cudaMemcpyKind kind = p->location == GLASSO_HOST ? cudaMemcpyHostToDevice
                                                           : cudaMemcpyDeviceToDevice;
    glasso_status s = work_ensure(w, n, st, err);
    if (s != GLASSO_OK) return s;
    if (p->input == GLASSO_INPUT_S) {
        CK(cudaMemcpyAsync(w.S, p->data, (size_t)(n * n) * sizeof(double), kind, st));
    } else {
        const int xb = p->dtype == GLASSO_F32 ? 4 : 8;
        s = work_ensure_x(w, p->m, n, xb, st, err);
        if (s != GLASSO_OK) return s;
        const void *X = p->data;
        if (p->location == GLASSO_HOST) {
            CK(cudaMemcpyAsync(w.Xraw, p->data, (size_t)(p->m * n) * xb, kind, st));
            X = w.Xraw;
        }
        s = form_S_ctx(w, st, precision, X, p->dtype, p->m, n, p->center, w.S, err);
        if (s != GLASSO_OK) return s;
    }
    s = check_symmetric(w, w.S, n, st, err);
    if (s != GLASSO_OK) return s;
    if (p->A0) {
        CK(cudaMemcpyAsync(w.A, p->A0, (size_t)(n * n) * sizeof(double), kind, st));
        s = check_symmetric(w, w.A, n, st, err);
        if (s != GLASSO_OK) return s;
    }
    return GLASSO_OK;
}

glasso_status validate(const glasso_problem *p) {
    if (!p || !p->data || p->n < 1 || !finite_pos(p->lambda) || !(p->tol >= 0.0)) return GLASSO_EINVAL;
    if (p->input != GLASSO_INPUT_S && p->input != GLASSO_INPUT_X) return GLASSO_EINVAL;
    if (p->location != GLASSO_HOST && p->location != GLASSO_DEVICE) return GLASSO_EINVAL;
    if (p->input == GLASSO_INPUT_X && (p->m < 1 || (p->dtype != GLASSO_F64 && p->dtype != GLASSO_F32)))
        return GLASSO_EINVAL;
    if (p->n > 46340) return GLASSO_EINVAL;  // n^2 int32-indexed pair bound
    if (p->inner != GLASSO_INNER_CD && p->inner != GLASSO_INNER_PCD_CG && p->inner != GLASSO_INNER_AUTO)
        return GLASSO_EINVAL;
    return GLASSO_OK;
}

glasso_status solve_one(Solver &sv, int64_t n, const glasso_problem *p, int mc, bool warm,
                        bool want_W, glasso_info *info, CoreSums *sums) {
    sv.inner = p->inner;
    return sv.precision == GLASSO_MIXED
               ? solve_core_mixed(sv, n, p->lambda, p->tol, mc, warm, p->one_level != 0,
                                  p->continuation != 0, info, sums)
               : solve_core(sv, n, p->lambda, p->tol, mc, warm, want_W, p->one_level != 0,
                            p->continuation != 0, info, sums);
}

// Exact screening (screen.cu): the isolated vertices of {|S_ij| > lambda} in
// closed form, every other vertex in one sub-problem on the principal
// sub-matrix of S (and of A0), solved like any problem and scattered back.
// The non-isolated components stay together: the relaxation never couples
// two components (A starts and stays block diagonal, so W does too, and a
// pair across components has A_ij = 0 and |G_ij| = |S_ij| <= lambda, so it
// never enters the free set).  Solving them together therefore reaches the
// same minimiser and pays the fixed cost of one solve, not one per component.
glasso_status solve_screened(Solver &sv, const glasso_problem *p, int mc, bool warm, bool want_W,
                             glasso_info *info) {
    Work &w = sv.w;
    cudaStream_t st = sv.st;
    std::string &err = sv.err;
    const int64_t n = p->n;
    const double lam = p->lambda;
    const size_t bytes = (size_t)n * (size_t)n * sizeof(double);
    glasso_status s = work_ensure_screen(w, n, st, err);
    if (s != GLASSO_OK) return s;
    CK(cudaMemcpyAsync(w.scr_S, w.S, bytes, cudaMemcpyDeviceToDevice, st));
    if (warm) CK(cudaMemcpyAsync(w.scr_A0, w.A, bytes, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(w.scr_A, 0, bytes, st));
    if (want_W) CK(cudaMemsetAsync(w.scr_W, 0, bytes, st));
    CK(cudaMemsetAsync(w.sc, 0, sizeof(DevScalars), st));
    CK(components(w.scr_S, n, lam, w.cc_parent, w.cc_comp, w.cc_size, &w.sc->cc_err, st));
    CK(screen_diag(w.scr_S, n, lam, w.cc_comp, w.cc_size, w.scr_A, want_W ? w.scr_W : nullptr,
                   w.scr_diag, &w.sc->err, st));
    std::vector<int32_t> comp((size_t)n);
    std::vector<double> diag((size_t)n);
    CK(cudaMemcpyAsync(comp.data(), w.cc_comp, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(diag.data(), w.scr_diag, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (sv.sync() != GLASSO_OK) return GLASSO_ECUDA;
    if (w.sc_host->cc_err) {
        err = "component labelling: a retry bound was exceeded";
        return GLASSO_ECUDA;
    }
    if (w.sc_host->err) return GLASSO_ENOTPD;
    // component sizes (a label is its component's smallest vertex)
    std::vector<int64_t> size((size_t)n, 0);
    for (int64_t i = 0; i < n; ++i) {
        const int32_t r = comp[i];
        if (r < 0 || r > i) {
            err = "component labelling: invalid label";
            return GLASSO_ECUDA;
        }
        ++size[r];
    }
    int64_t ncomp = 0, max_block = 0;
    for (int64_t r = 0; r < n; ++r)
        if (size[r]) {
            ++ncomp;
            max_block = std::max(max_block, size[r]);
        }
    // isolated vertices: F, log det and ||A||_1 of A_ii = 1/(S_ii + lambda), in
    // index order; the other vertices, ascending, form the sub-problem
    std::vector<int32_t> idx;
    idx.reserve((size_t)n);
    double F = 0.0, logdet = 0.0, l1 = 0.0;
    int64_t n_iso = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (size[comp[i]] == 1) {
            const double d = diag[i] + lam;
            F += log(d) + 1.0;  // -log(1/d) + (S_ii + lambda)/d
            logdet -= log(d);
            l1 += 1.0 / d;
            ++n_iso;
        } else {
            idx.push_back((int32_t)i);
        }
    }
    const int64_t nb = (int64_t)idx.size();
    glasso_info sub;
    memset(&sub, 0, sizeof(sub));
    sub.status = GLASSO_OK;
    double kkt_sum = 0.0;
    if (nb > 0) {
        CoreSums cs;
        CK(cudaMemcpyAsync(w.scr_idx, idx.data(), (size_t)nb * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        CK(gather_block(w.scr_S, n, w.scr_idx, nb, w.S, st));
        if (warm) CK(gather_block(w.scr_A0, n, w.scr_idx, nb, w.A, st));
        s = solve_one(sv, nb, p, mc, warm, want_W, &sub, &cs);
        if (s == GLASSO_ECUDA || s == GLASSO_ENOTPD) return s;
        CK(scatter_block(w.A, nb, w.scr_idx, n, w.scr_A, st));
        if (want_W) CK(scatter_block(w.W, nb, w.scr_idx, n, w.scr_W, st));
        F += sub.objective;
        logdet += sub.logdet;
        kkt_sum = sub.rel_kkt * cs.l1;  // the isolated vertices are exact: no residual
        l1 += cs.l1;
    }
    CK(cudaMemcpyAsync(w.A, w.scr_A, bytes, cudaMemcpyDeviceToDevice, st));
    if (want_W) CK(cudaMemcpyAsync(w.W, w.scr_W, bytes, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(w.S, w.scr_S, bytes, cudaMemcpyDeviceToDevice, st));
    if (info) {
        *info = sub;
        info->objective = F;
        info->logdet = logdet;
        info->rel_kkt = l1 > 0.0 ? kkt_sum / l1 : 0.0;
        info->nnz = sub.nnz + n_iso;
        info->max_nnz = sub.max_nnz + n_iso;
        info->components = ncomp;
        info->max_block = max_block;
    }
    return (glasso_status)sub.status;
}

glasso_status solve_in(Work &w, cudaStream_t st, size_t budget, const glasso_problem *p,
                       double *A_out, double *W_out, glasso_info *info, std::string &err,
                       Prof *prof, bool reuse_A, int out_location, int precision) {
    auto t0 = std::chrono::steady_clock::now();
    glasso_info loc;
    memset(&loc, 0, sizeof(loc));
    glasso_status s = validate(p);
    if (s == GLASSO_OK && !A_out) s = GLASSO_EINVAL;
    if (s == GLASSO_OK && budget) {
        const int64_t m = p->input == GLASSO_INPUT_X ? p->m : 0;
        if (footprint(p->n, m, p->dtype == GLASSO_F32 ? 4 : 8, p->screen != 0) > budget) s = GLASSO_ENOMEM;
    }
    if (s == GLASSO_OK) {
        glasso_problem q = *p;
        if (reuse_A) q.A0 = nullptr;
        s = stage_problem(w, st, &q, err, precision);
    }
    if (s == GLASSO_OK) {
        Solver sv{w, st, err, prof, precision};
        const int mc = p->max_cycles > 0 ? p->max_cycles : 200;
        const bool warm = p->A0 != nullptr || reuse_A;
        s = p->screen ? solve_screened(sv, p, mc, warm, W_out != nullptr, &loc)
                      : solve_one(sv, p->n, p, mc, warm, W_out != nullptr, &loc, nullptr);
        if (s != GLASSO_ECUDA && s != GLASSO_ENOTPD && s != GLASSO_ETIMEOUT) {
            const cudaMemcpyKind kind = out_location == GLASSO_HOST ? cudaMemcpyDeviceToHost
                                                                    : cudaMemcpyDeviceToDevice;
            const size_t bytes = (size_t)(p->n * p->n) * sizeof(double);
            cudaError_t e = cudaMemcpyAsync(A_out, w.A, bytes, kind, st);
            if (e == cudaSuccess && W_out) e = cudaMemcpyAsync(W_out, w.W, bytes, kind, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) s = fail_cuda(err, e, "copy out");
        }
        if (prof) prof_collect(prof);
    }
    loc.status = s;
    loc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = loc;
    return s;
}

// ---- serving --------------------------------------------------------------
struct Request {
    uint64_t ticket = 0;
    glasso_problem p{};
    std::vector<char> data;
    std::vector<double> a0;
    double *A_out = nullptr;
    int out_location = GLASSO_HOST;
    glasso_info info{};
    glasso_status status = GLASSO_EAGAIN;
    size_t fp = 0;
    bool done = false;
    // a lambda path on the same data: solved after p, in order, each warm
    // started from the previous solution in the worker's workspace
    std::vector<glasso_problem> more;
    std::vector<double *> more_out;
    std::vector<glasso_info> more_info;
};

struct Serve {
    glasso_ctx *ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> all;
    std::vector<std::thread> workers;
    size_t reserved = 0;
    uint64_t next = 1;
    bool stop = false;
};

int serve_slots() {
    const char *e = getenv("GLASSO_SERVE_SLOTS");
    int k = e ? atoi(e) : 4;
    return k < 1 ? 1 : (k > 64 ? 64 : k);
}

void worker_main(Serve *sv) {
    cudaSetDevice(sv->ctx->device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    Work w;
    w.dag_share = serve_slots();  // the slots' solves share the GPU
    std::string err;
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] {
                if (sv->stop) return true;
                if (sv->queue.empty()) return false;
                // admission: the head request must fit the remaining budget
                const size_t b = sv->ctx->budget;
                return b == 0 || sv->reserved == 0 || sv->reserved + sv->queue.front()->fp <= b;
            });
            if (sv->stop) break;
            r = sv->queue.front();
            sv->queue.pop_front();
            sv->reserved += r->fp;
        }
        if (w.cap_n > 0 && (w.cap_n < r->p.n || w.cap_n > 2 * r->p.n)) work_free(w, st);
        glasso_info info;
        glasso_status s = solve_in(w, st, 0, &r->p, r->A_out, nullptr, &info, err, nullptr, false,
                                   r->out_location, sv->ctx->precision);
        for (size_t i = 0; i < r->more.size(); ++i) {
            glasso_info inf2;
            memset(&inf2, 0, sizeof(inf2));
            glasso_status s2 = GLASSO_ECUDA;
            if (s == GLASSO_OK || s == GLASSO_EMAXITER || s == GLASSO_ELINESEARCH) {
                s2 = solve_in(w, st, 0, &r->more[i], r->more_out[i], nullptr, &inf2, err, nullptr,
                              true, r->out_location, sv->ctx->precision);
            } else {
                inf2.status = s;
            }
            r->more_info[i] = inf2;
            if (s == GLASSO_OK) s = s2;
        }
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            r->info = info;
            r->status = s;
            r->done = true;
            sv->reserved -= r->fp;
            r->data.clear();
            r->data.shrink_to_fit();
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
    work_free(w, st);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
}

Serve *serve_get(glasso_ctx *ctx) {
    if (!ctx->serve) {
        Serve *s = new Serve();
        s->ctx = ctx;
        const int k = serve_slots();
        for (int i = 0; i < k; ++i) s->workers.emplace_back(worker_main, s);
        ctx->serve = s;
    }
    return (Serve *)ctx->serve;
}

void serve_shutdown(glasso_ctx *ctx) {
    Serve *s = (Serve *)ctx->serve;
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    for (auto &kv : s->all) delete kv.second;
    delete s;
    ctx->serve = nullptr;
}


// Queue `count` problems on the same data (count > 1: a warm-started lambda
// path) as one request; the input is copied to the host before returning.
glasso_status submit_chain(glasso_ctx *ctx, const glasso_problem *p, int count, double **A_out,
                           uint64_t *ticket) {
    if (!ctx || !ticket || !A_out || count < 1) return GLASSO_EINVAL;
    for (int k = 0; k < count; ++k) {
        glasso_status s = validate(&p[k]);
        if (s != GLASSO_OK) return s;
        if (!A_out[k]) return GLASSO_EINVAL;
    }
    const int64_t m = p->input == GLASSO_INPUT_X ? p->m : 0;
    const int xb = p->dtype == GLASSO_F32 ? 4 : 8;
    bool screen = false;
    for (int k = 0; k < count; ++k) screen = screen || p[k].screen != 0;
    const size_t fp = footprint(p->n, m, xb, screen);
    if (ctx->budget && fp > ctx->budget) return GLASSO_ENOMEM;
    Request *r = new Request();
    r->p = *p;
    const size_t bytes = p->input == GLASSO_INPUT_S ? (size_t)(p->n * p->n) * 8 : (size_t)(m * p->n) * xb;
    r->data.resize(bytes);
    const cudaMemcpyKind kind = p->location == GLASSO_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
    cudaSetDevice(ctx->device);
    if (cudaMemcpy(r->data.data(), p->data, bytes, kind) != cudaSuccess) {
        delete r;
        return GLASSO_ECUDA;
    }
    if (p->A0) {
        r->a0.resize((size_t)(p->n * p->n));
        if (cudaMemcpy(r->a0.data(), p->A0, r->a0.size() * 8, kind) != cudaSuccess) {
            delete r;
            return GLASSO_ECUDA;
        }
        r->p.A0 = r->a0.data();
    }
    // the staged copies live on the host; outputs go where the caller said
    r->p.data = r->data.data();
    r->A_out = A_out[0];
    r->out_location = p->location;
    r->fp = fp;
    r->p.location = GLASSO_HOST;  // inputs now live in the request's host copy
    for (int k = 1; k < count; ++k) {
        glasso_problem q = p[k];
        q.data = r->data.data();
        q.location = GLASSO_HOST;
        q.A0 = nullptr;
        r->more.push_back(q);
        r->more_out.push_back(A_out[k]);
    }
    r->more_info.resize(r->more.size());
    Serve *sv = serve_get(ctx);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r->ticket = sv->next++;
        sv->all[r->ticket] = r;
        sv->queue.push_back(r);
    }
    sv->cv_work.notify_one();
    *ticket = r->ticket;
    return GLASSO_OK;
}

// Wait for a request; infos[0 .. 1 + more) receive its problems' infos.
glasso_status wait_chain(glasso_ctx *ctx, uint64_t ticket, glasso_info *infos) {
    Serve *sv = (Serve *)ctx->serve;
    if (!sv) return GLASSO_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return GLASSO_EINVAL;
    Request *r = it->second;
    sv->cv_done.wait(lk, [&] { return r->done; });
    if (infos) {
        infos[0] = r->info;
        for (size_t i = 0; i < r->more_info.size(); ++i) infos[1 + i] = r->more_info[i];
    }
    glasso_status s = r->status;
    sv->all.erase(it);
    delete r;
    return s;
}
}  // namespace

// =================================================================== C ABI
extern "C" {

const char *glasso_strerror(glasso_status s) {
    switch (s) {
        case GLASSO_OK: return "ok";
        case GLASSO_EINVAL: return "invalid argument";
        case GLASSO_ENOMEM: return "out of device memory or over budget";
        case GLASSO_ENOTPD: return "initial iterate not positive definite";
        case GLASSO_ELINESEARCH: return "line search failed";
        case GLASSO_EMAXITER: return "maximum number of cycles reached";
        case GLASSO_EAGAIN: return "not finished";
        case GLASSO_ETIMEOUT: return "timed out";
        case GLASSO_ECUDA: return "CUDA error";
    }
    return "unknown status";
}

glasso_status glasso_create(const glasso_config *cfg, glasso_ctx **out) {
    if (!out) return GLASSO_EINVAL;
    *out = nullptr;
    if (!cfg || (cfg->precision != GLASSO_FP64 && cfg->precision != GLASSO_MIXED)) return GLASSO_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev)
        return GLASSO_ECUDA;
    if (cudaSetDevice(cfg->device) != cudaSuccess) return GLASSO_ECUDA;
    glasso_ctx *c = new glasso_ctx();
    c->device = cfg->device;
    c->precision = cfg->precision;
    c->budget = cfg->mem_budget_bytes;
    if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return GLASSO_ECUDA;
    }
    c->stream = c->own_stream;
    *out = c;
    return GLASSO_OK;
}

void glasso_destroy(glasso_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    serve_shutdown(ctx);
    work_free(ctx->w, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->prof) delete (Prof *)ctx->prof;
    cudaStreamDestroy(ctx->own_stream);
    delete ctx;
}

glasso_status glasso_set_stream(glasso_ctx *ctx, void *stream) {
    if (!ctx) return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
    return GLASSO_OK;
}

const char *glasso_last_error(glasso_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

glasso_status glasso_set_profiling(glasso_ctx *ctx, int on) {
    if (!ctx) return GLASSO_EINVAL;
    if (!ctx->prof) ctx->prof = new Prof();
    Prof *p = (Prof *)ctx->prof;
    p->on = on != 0;
    return GLASSO_OK;
}

glasso_status glasso_get_profile(glasso_ctx *ctx, glasso_profile *out, int reset) {
    if (!ctx || !out) return GLASSO_EINVAL;
    memset(out, 0, sizeof(*out));
    if (!ctx->prof) ctx->prof = new Prof();
    Prof *p = (Prof *)ctx->prof;
    for (int c = 0; c < GLASSO_PROF_CLASSES; ++c) {
        out->ms[c] = p->ms[c];
        out->launches[c] = p->count[c];
        out->work[c] = p->work[c];
        if (reset) { p->ms[c] = 0; p->count[c] = 0; p->work[c] = 0; }
    }
    out->kernels = g_launches.load() - p->kernels_base;
    if (reset) p->kernels_base = g_launches.load();
    for (int k = 0; k < GLASSO_PATHS; ++k) {
        const long long v = g_paths[k].load();
        out->paths[k] = v - p->paths_base[k];
        if (reset) p->paths_base[k] = v;
    }
    return GLASSO_OK;
}

glasso_status glasso_set_debug(glasso_ctx *ctx, int knob, int64_t value) {
    if (!ctx) return GLASSO_EINVAL;
    Work &w = ctx->w;
    switch (knob) {
        case GLASSO_DEBUG_WAIT_CYCLES:
            if (value < 0) return GLASSO_EINVAL;
            w.dbg_wait_cycles = (long long)value;
            return GLASSO_OK;
        case GLASSO_DEBUG_WAIT_UNREACHABLE: w.dbg_wait_unreachable = value != 0; return GLASSO_OK;
        case GLASSO_DEBUG_LS_REJECT: w.dbg_ls_reject = value != 0; return GLASSO_OK;
        case GLASSO_DEBUG_TC_DAG_TILES:
            if (value < 0 || value > 32) return GLASSO_EINVAL;
            w.dbg_dag_tiles = (int)value;
            return GLASSO_OK;
        default: return GLASSO_EINVAL;
    }
}

glasso_status glasso_solve(glasso_ctx *ctx, const glasso_problem *p, double *A_out, double *W_out,
                           glasso_info *info) {
    if (!ctx) return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    return solve_in(ctx->w, ctx->stream, ctx->budget, p, A_out, W_out, info, ctx->last_error,
                    (Prof *)ctx->prof, false, p ? p->location : GLASSO_HOST, ctx->precision);
}

glasso_status glasso_solve_batch(glasso_ctx *ctx, const glasso_problem *p, int count,
                                 int warm_from_prev, double **A_out, glasso_info *infos) {
    if (!ctx || !p || count < 0 || (count > 0 && !A_out)) return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    glasso_status first = GLASSO_OK;
    if (!warm_from_prev) {
        // independent problems: run them concurrently through the serving slots
        std::vector<uint64_t> tickets(count);
        for (int k = 0; k < count; ++k) {
            glasso_status s = glasso_submit(ctx, &p[k], A_out[k], &tickets[k]);
            if (s != GLASSO_OK) {
                if (infos) { memset(&infos[k], 0, sizeof(glasso_info)); infos[k].status = s; }
                if (first == GLASSO_OK) first = s;
                tickets[k] = 0;
            }
        }
        for (int k = 0; k < count; ++k) {
            if (!tickets[k]) continue;
            glasso_info inf;
            glasso_status s;
            while ((s = glasso_poll(ctx, tickets[k], 1000000, &inf)) == GLASSO_EAGAIN) {}
            if (infos) infos[k] = inf;
            if (s != GLASSO_OK && first == GLASSO_OK) first = s;
        }
        return first;
    }
    // lambda paths: maximal runs of problems on the same data; several runs go
    // through the serving slots concurrently (each run in order on one slot)
    auto continues = [&](int k) {
        return k > 0 && p[k].A0 == nullptr && p[k].n == p[k - 1].n && p[k].data == p[k - 1].data &&
               p[k].input == p[k - 1].input;
    };
    std::vector<int> starts;
    for (int k = 0; k < count; ++k)
        if (!continues(k)) starts.push_back(k);
    if (starts.size() > 1) {
        std::vector<uint64_t> tickets(starts.size(), 0);
        for (size_t c = 0; c < starts.size(); ++c) {
            const int k0 = starts[c];
            const int k1 = c + 1 < starts.size() ? starts[c + 1] : count;
            glasso_status s = submit_chain(ctx, &p[k0], k1 - k0, &A_out[k0], &tickets[c]);
            if (s != GLASSO_OK) {
                for (int k = k0; k < k1; ++k)
                    if (infos) { memset(&infos[k], 0, sizeof(glasso_info)); infos[k].status = s; }
                if (first == GLASSO_OK) first = s;
            }
        }
        for (size_t c = 0; c < starts.size(); ++c) {
            if (!tickets[c]) continue;
            const int k0 = starts[c];
            const int k1 = c + 1 < starts.size() ? starts[c + 1] : count;
            std::vector<glasso_info> inf(k1 - k0);
            glasso_status s = wait_chain(ctx, tickets[c], inf.data());
            if (infos)
                for (int k = k0; k < k1; ++k) infos[k] = inf[k - k0];
            if (s != GLASSO_OK && first == GLASSO_OK) first = s;
        }
        return first;
    }
    for (int k = 0; k < count; ++k) {
        const bool chain = continues(k);
        glasso_info inf;
        glasso_status s;
        if (chain) {
            // continue from the previous solution kept in the workspace (w.A)
            s = solve_in(ctx->w, ctx->stream, ctx->budget, &p[k], A_out[k], nullptr, &inf,
                         ctx->last_error, (Prof *)ctx->prof, true, p[k].location, ctx->precision);
        } else {
            s = solve_in(ctx->w, ctx->stream, ctx->budget, &p[k], A_out[k], nullptr, &inf,
                         ctx->last_error, (Prof *)ctx->prof, false, p[k].location, ctx->precision);
        }
        if (infos) infos[k] = inf;
        if (s != GLASSO_OK && first == GLASSO_OK) first = s;
    }
    return first;
}

// The batched solver in one persistent launch (fused.cu): the inputs of every
// path are staged (S copied, or formed from X), the launch runs all solves,
// then the solutions and statistics are copied out.
glasso_status glasso_solve_batch_fused(glasso_ctx *ctx, const glasso_problem *p, int count,
                                       int warm_from_prev, double **A_out, glasso_info *infos) {
    if (!ctx || !p || count < 0 || (count > 0 && !A_out)) return GLASSO_EINVAL;
    if (count == 0) return GLASSO_OK;
    cudaSetDevice(ctx->device);
    Work &w = ctx->w;
    cudaStream_t st = ctx->stream;
    std::string &err = ctx->last_error;
    auto fail_all = [&](glasso_status s) {
        if (infos)
            for (int k = 0; k < count; ++k) {
                memset(&infos[k], 0, sizeof(glasso_info));
                infos[k].status = s;
            }
        return s;
    };
    int nmax = 0;
    for (int k = 0; k < count; ++k) {
        const glasso_problem &q = p[k];
        if (validate(&q) != GLASSO_OK || q.n > GLASSO_FUSED_MAX_N || q.screen || q.continuation ||
            q.inner == GLASSO_INNER_PCD_CG || !A_out[k])
            return fail_all(GLASSO_EINVAL);
        nmax = std::max(nmax, (int)q.n);
    }
    // paths: maximal runs continuing one another (the rule of glasso_solve_batch)
    auto continues = [&](int k) {
        return warm_from_prev && k > 0 && p[k].A0 == nullptr && p[k].n == p[k - 1].n &&
               p[k].data == p[k - 1].data && p[k].input == p[k - 1].input;
    };
    std::vector<int2> paths;
    for (int k = 0; k < count; ++k) {
        if (!continues(k)) paths.push_back(make_int2(k, k + 1));
        else paths.back().y = k + 1;
    }
    const int npaths = (int)paths.size();
    // longest first: the device queue hands them out in this order
    std::stable_sort(paths.begin(), paths.end(), [&](const int2 &a, const int2 &b) {
        const double ca = std::pow((double)p[a.x].n, 3.0) * (a.y - a.x);
        const double cb = std::pow((double)p[b.x].n, 3.0) * (b.y - b.x);
        return ca > cb;
    });
    int dev = 0, nsm = 1;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::min(npaths, nsm);
    // one device arena: S per path, A per problem (A0 staged there), the
    // problem and result records, the paths, the queue counter, the slots
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t off = 0;
    std::vector<size_t> s_off(npaths), a_off(count);
    for (int c = 0; c < npaths; ++c) {
        s_off[c] = off;
        off += al((size_t)p[paths[c].x].n * p[paths[c].x].n * sizeof(double));
    }
    for (int k = 0; k < count; ++k) {
        a_off[k] = off;
        off += al((size_t)p[k].n * p[k].n * sizeof(double));
    }
    const size_t prob_off = off;
    off += al((size_t)count * sizeof(FusedProblem));
    const size_t res_off = off;
    off += al((size_t)count * sizeof(FusedResult));
    const size_t path_off = off;
    off += al((size_t)npaths * sizeof(int2));
    const size_t next_off = off;
    off += 256;
    const size_t slot = fused_slot_bytes(nmax);
    const size_t arena_off = off;
    off += (size_t)grid * slot;
    if (ctx->budget && off > ctx->budget) return fail_all(GLASSO_ENOMEM);
    glasso_status s0 = work_ensure(w, 1, st, err);
    if (s0 != GLASSO_OK) return fail_all(s0);
    char *base = nullptr;
    if (cudaMallocAsync((void **)&base, off, st) != cudaSuccess) {
        cudaGetLastError();
        return fail_all(GLASSO_ENOMEM);
    }
    struct Free {
        char *p;
        cudaStream_t st;
        ~Free() { cudaFreeAsync(p, st); }
    } guard{base, st};
    // stage the inputs
    for (int c = 0; c < npaths; ++c) {
        const glasso_problem &q = p[paths[c].x];
        const int64_t n = q.n;
        double *Sd = (double *)(base + s_off[c]);
        const cudaMemcpyKind kind = q.location == GLASSO_HOST ? cudaMemcpyHostToDevice
                                                              : cudaMemcpyDeviceToDevice;
        if (q.input == GLASSO_INPUT_S) {
            CK(cudaMemcpyAsync(Sd, q.data, (size_t)(n * n) * sizeof(double), kind, st));
            glasso_status s = check_symmetric(w, Sd, n, st, err);
            if (s != GLASSO_OK) return fail_all(s);
        } else {
            const int xb = q.dtype == GLASSO_F32 ? 4 : 8;
            glasso_status s = work_ensure_x(w, q.m, n, xb, st, err);
            if (s != GLASSO_OK) return fail_all(s);
            const void *X = q.data;
            if (q.location == GLASSO_HOST) {
                CK(cudaMemcpyAsync(w.Xraw, q.data, (size_t)(q.m * n) * xb, kind, st));
                X = w.Xraw;
            }
            CK(form_S(X, q.dtype, q.m, n, q.center, Sd, w.Xin, st));
        }
    }
    std::vector<FusedProblem> fp(count);
    for (int c = 0; c < npaths; ++c)
        for (int k = paths[c].x; k < paths[c].y; ++k) {
            const glasso_problem &q = p[k];
            FusedProblem &f = fp[k];
            f.S = (const double *)(base + s_off[c]);
            f.A_out = (double *)(base + a_off[k]);
            f.A0 = nullptr;
            if (q.A0) {
                const cudaMemcpyKind kind = q.location == GLASSO_HOST ? cudaMemcpyHostToDevice
                                                                      : cudaMemcpyDeviceToDevice;
                CK(cudaMemcpyAsync(f.A_out, q.A0, (size_t)q.n * q.n * sizeof(double), kind, st));
                glasso_status s = check_symmetric(w, f.A_out, q.n, st, err);
                if (s != GLASSO_OK) return fail_all(s);
                f.A0 = f.A_out;
            }
            f.lambda = q.lambda;
            f.tol = q.tol;
            f.n = (int)q.n;
            f.max_cycles = q.max_cycles > 0 ? q.max_cycles : 200;
            f.one_level = q.one_level != 0;
            f.pad = 0;
        }
    FusedProblem *dprob = (FusedProblem *)(base + prob_off);
    FusedResult *dres = (FusedResult *)(base + res_off);
    int2 *dpath = (int2 *)(base + path_off);
    CK(cudaMemcpyAsync(dprob, fp.data(), (size_t)count * sizeof(FusedProblem), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dpath, paths.data(), (size_t)npaths * sizeof(int2), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(dres, 0, (size_t)count * sizeof(FusedResult), st));
    CK(fused_paths(dprob, dres, dpath, npaths, (int *)(base + next_off), base + arena_off, slot, nmax, grid,
                   st));
    path_hit(GLASSO_PATH_FUSED, count);
    std::vector<FusedResult> res(count);
    CK(cudaMemcpyAsync(res.data(), dres, (size_t)count * sizeof(FusedResult), cudaMemcpyDeviceToHost, st));
    for (int k = 0; k < count; ++k) {
        const cudaMemcpyKind kind = p[k].location == GLASSO_HOST ? cudaMemcpyDeviceToHost
                                                                 : cudaMemcpyDeviceToDevice;
        CK(cudaMemcpyAsync(A_out[k], base + a_off[k], (size_t)p[k].n * p[k].n * sizeof(double), kind, st));
    }
    CK(cudaStreamSynchronize(st));
    // with profiling on, the step classes receive the CTAs' summed device time
    if (ctx->prof && ((Prof *)ctx->prof)->on) {
        Prof *pr = (Prof *)ctx->prof;
        for (int k = 0; k < count; ++k)
            for (int c = 0; c < FUSED_CLASSES; ++c) pr->ms[c] += res[k].cls_ns[c] * 1e-6;
    }
    glasso_status first = GLASSO_OK;
    for (int k = 0; k < count; ++k) {
        const FusedResult &r = res[k];
        if (infos) {
            glasso_info &inf = infos[k];
            memset(&inf, 0, sizeof(glasso_info));
            inf.status = r.status;
            inf.cycles = r.cycles;
            inf.relaxations = r.relaxations;
            inf.ls_trials = r.ls_trials;
            inf.objective = r.objective;
            inf.rel_kkt = r.rel_kkt;
            inf.max_kkt = r.max_kkt;
            inf.logdet = r.logdet;
            inf.seconds = r.t1 >= r.t0 ? (double)(r.t1 - r.t0) * 1e-9 : 0.0;
            inf.nnz = r.nnz;
            inf.max_nnz = r.max_nnz;
            inf.inner_iters = r.sweeps;
            inf.flops = r.flops;
        }
        if (r.status != GLASSO_OK && first == GLASSO_OK) first = (glasso_status)r.status;
    }
    return first;
}

glasso_status glasso_submit(glasso_ctx *ctx, const glasso_problem *p, double *A_out,
                            uint64_t *ticket) {
    return submit_chain(ctx, p, 1, &A_out, ticket);
}

glasso_status glasso_poll(glasso_ctx *ctx, uint64_t ticket, int64_t timeout_us, glasso_info *info) {
    if (!ctx || !ctx->serve) return GLASSO_EINVAL;
    Serve *sv = (Serve *)ctx->serve;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return GLASSO_EINVAL;
    Request *r = it->second;
    if (!r->done && timeout_us > 0)
        sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; });
    if (!r->done) return GLASSO_EAGAIN;
    if (info) *info = r->info;
    glasso_status s = r->status;
    sv->all.erase(it);
    delete r;
    return s;
}

// ---- step-level entry points ----------------------------------------------
#define CTX_CK(call)                                                          \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return fail_cuda(ctx->last_error, e_, #call); \
    } while (0)

static glasso_status sync_ctx(glasso_ctx *ctx) {
    CTX_CK(cudaMemcpyAsync(ctx->w.sc_host, ctx->w.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                           ctx->stream));
    CTX_CK(cudaStreamSynchronize(ctx->stream));
    return GLASSO_OK;
}

glasso_status glasso_form_S(glasso_ctx *ctx, const void *X, int dtype, int64_t m, int64_t n,
                            int center, double *S) {
    if (!ctx || !X || !S || m < 1 || n < 1 || (dtype != GLASSO_F64 && dtype != GLASSO_F32))
        return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    glasso_status s = work_ensure(ctx->w, 1, ctx->stream, ctx->last_error);
    if (s == GLASSO_OK) s = work_ensure_x(ctx->w, m, n, 0, ctx->stream, ctx->last_error);
    if (s != GLASSO_OK) return s;
    s = form_S_ctx(ctx->w, ctx->stream, ctx->precision, X, dtype, m, n, center, S, ctx->last_error);
    if (s != GLASSO_OK) return s;
    CTX_CK(cudaStreamSynchronize(ctx->stream));
    return GLASSO_OK;
}

glasso_status glasso_potrf(glasso_ctx *ctx, double *A, int64_t n, int *info, double *logdet) {
    if (!ctx || !A || n < 1) return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    glasso_status s = work_ensure(ctx->w, n, ctx->stream, ctx->last_error);
    if (s != GLASSO_OK) return s;
    Prof *prof = (Prof *)ctx->prof;
    Solver sv{ctx->w, ctx->stream, ctx->last_error, prof};
    cudaEvent_t eb;
    sv.mark_begin(0, eb);
    CTX_CK(potrf(A, n, ctx->w.xd, ctx->w.ldiag, ctx->w.sc, ctx->stream));
    sv.mark_end(0, eb, (double)n * n * n / 3.0);
    s = sync_ctx(ctx);
    if (prof) prof_collect(prof);
    if (s != GLASSO_OK) return s;
    if (info) *info = ctx->w.sc_host->info;
    if (logdet) *logdet = ctx->w.sc_host->logdet;
    return GLASSO_OK;
}

glasso_status glasso_inverse(glasso_ctx *ctx, const double *L, int64_t n, double *W) {
    if (!ctx || !L || !W || n < 1) return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    glasso_status s = work_ensure(ctx->w, n, ctx->stream, ctx->last_error);
    if (s != GLASSO_OK) return s;
    Prof *prof = (Prof *)ctx->prof;
    Solver sv{ctx->w, ctx->stream, ctx->last_error, prof};
    cudaEvent_t eb;
    sv.mark_begin(1, eb);
    CTX_CK(inverse(L, n, W, ctx->w.T, ctx->w.U, ctx->stream));
    sv.mark_end(1, eb, 2.0 * (double)n * n * n / 3.0);
    CTX_CK(cudaStreamSynchronize(ctx->stream));
    if (prof) prof_collect(prof);
    return GLASSO_OK;
}

// BCD-IC's Schur-complement line-search log det (bcd.cu pieces, dense.cu's
// FP64 factorisation and inverse) for the block with index lists i1 (I) and
// i2 (the others); inI: the block's mask on the device.  Uses w.T, w.U, w.xd,
// w.ldiag and w.sc; synchronises the stream.
static glasso_status bcd_logdet_dev(glasso_ctx *ctx, const double *A, int64_t n, const int32_t *pi,
                                    const int32_t *pj, int64_t np, const double *D, const uint8_t *inI,
                                    const std::vector<int32_t> &i1, const std::vector<int32_t> &i2,
                                    double alpha, double *logdet, int *code) {
    Work &w = ctx->w;
    cudaStream_t st = ctx->stream;
    const int64_t m1 = (int64_t)i1.size(), m2 = (int64_t)i2.size();
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t nn = (size_t)n * n;
    const size_t o_dl = 0, o_a22 = o_dl + al(nn * 8), o_inv = o_a22 + al((size_t)(m2 * m2) * 8),
                 o_y = o_inv + al((size_t)(m2 * m2) * 8), o_z = o_y + al((size_t)(m2 * m1) * 8),
                 o_m = o_z + al((size_t)(m2 * m1) * 8), o_i1 = o_m + al((size_t)(m1 * m1) * 8),
                 o_i2 = o_i1 + al((size_t)m1 * 4), o_bad = o_i2 + al((size_t)m2 * 4), total = o_bad + 256;
    char *base = nullptr;
    if (cudaMallocAsync((void **)&base, total, st) != cudaSuccess) {
        cudaGetLastError();
        return GLASSO_ENOMEM;
    }
    struct Free {
        char *p;
        cudaStream_t st;
        ~Free() { cudaFreeAsync(p, st); }
    } guard{base, st};
    double *Dl = (double *)(base + o_dl), *A22 = (double *)(base + o_a22), *Ainv = (double *)(base + o_inv);
    double *Y = (double *)(base + o_y), *Z = (double *)(base + o_z), *M = (double *)(base + o_m);
    int32_t *d1 = (int32_t *)(base + o_i1), *d2 = (int32_t *)(base + o_i2);
    int *bad = (int *)(base + o_bad);
    CTX_CK(cudaMemsetAsync(Dl, 0, nn * 8, st));
    CTX_CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
    if (m1) CTX_CK(cudaMemcpyAsync(d1, i1.data(), (size_t)m1 * 4, cudaMemcpyHostToDevice, st));
    if (m2) CTX_CK(cudaMemcpyAsync(d2, i2.data(), (size_t)m2 * 4, cudaMemcpyHostToDevice, st));
    CTX_CK(bcd_scatter(pi, pj, D, np, n, inI, Dl, bad, st));
    int hbad = 0;
    CTX_CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    CTX_CK(cudaStreamSynchronize(st));
    if (hbad == 2) return GLASSO_EINVAL;
    if (hbad == 1) {
        *code = -1;
        return GLASSO_OK;
    }
    double ld22 = 0.0;
    glasso_status s;
    if (m2 > 0) {
        CTX_CK(bcd_gather(A, n, d2, m2, A22, st));
        CTX_CK(potrf(A22, m2, w.xd, w.ldiag, w.sc, st));
        s = sync_ctx(ctx);
        if (s != GLASSO_OK) return s;
        if (w.sc_host->info != 0) {
            *code = 1;
            return GLASSO_OK;
        }
        ld22 = w.sc_host->logdet;
        CTX_CK(inverse(A22, m2, Ainv, w.T, w.U, st));
        CTX_CK(bcd_solve(Ainv, m2, A, Dl, n, d1, m1, d2, Y, Z, st));
    }
    double ld = ld22;
    if (m1 > 0) {
        CTX_CK(bcd_assemble(A, Dl, n, d1, m1, d2, m2, Y, Z, alpha, M, st));
        CTX_CK(potrf(M, m1, w.xd, w.ldiag, w.sc, st));
        s = sync_ctx(ctx);
        if (s != GLASSO_OK) return s;
        if (w.sc_host->info != 0) {
            *code = 2;
            return GLASSO_OK;
        }
        ld += w.sc_host->logdet;
    }
    CTX_CK(cudaStreamSynchronize(st));
    *code = 0;
    if (logdet) *logdet = ld;
    return GLASSO_OK;
}

glasso_status glasso_bcd_logdet(glasso_ctx *ctx, const double *A, int64_t n, const int32_t *pi,
                                const int32_t *pj, int64_t np, const double *D, const uint8_t *inI,
                                double alpha, double *logdet, int *code) {
    if (!ctx || !A || !inI || !code || n < 1 || np < 0 || (np > 0 && (!pi || !pj || !D)) ||
        !isfinite(alpha))
        return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    glasso_status s = work_ensure(ctx->w, n, ctx->stream, ctx->last_error);
    if (s != GLASSO_OK) return s;
    std::vector<uint8_t> mask((size_t)n);
    CTX_CK(cudaMemcpyAsync(mask.data(), inI, (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
    CTX_CK(cudaStreamSynchronize(ctx->stream));
    std::vector<int32_t> i1, i2;
    for (int64_t i = 0; i < n; ++i) (mask[i] ? i1 : i2).push_back((int32_t)i);
    return bcd_logdet_dev(ctx, A, n, pi, pj, np, D, inI, i1, i2, alpha, logdet, code);
}

// One BCD-IC iteration (Algorithm 2) with every block step on the device: per
// block of consecutive columns, W from the FP64 factorisation, the block's
// free set by the candidate scan over its pairs, the Newton direction (CD
// sweeps or PCD-CG), the line search over the samples alpha = 2^-t with log
// det(A + alpha Delta) from the Schur complement.  The block loop and the
// sample decisions run on the host.
// The iteration itself.  cand_i/cand_j (host, optional): the candidates the
// block free sets are taken from (the ML-cycle's C_l), else all pairs.  The
// block's candidates live in buffers of their own, so the fine free set and
// the level tags of the workspace are left untouched.
static glasso_status bcd_iteration_impl(glasso_ctx *ctx, const double *S, double *A, int64_t n, double lambda,
                                        int64_t block, int inner, int nsweeps, int rule,
                                        const std::vector<int32_t> *cand_i, const std::vector<int32_t> *cand_j,
                                        double *F_out, int *moved, int *trials) {
    if (block == 0 || block > n) block = n;
    Work &w = ctx->w;
    cudaStream_t st = ctx->stream;
    glasso_status s = work_ensure(w, n, st, ctx->last_error);
    if (s != GLASSO_OK) return s;
    // the mask and two candidate lists of at most block * n pairs
    const size_t capc = (size_t)block * (size_t)n + 1;
    char *base = nullptr;
    const size_t o_c1 = ((size_t)n + 255) & ~(size_t)255, o_c2 = o_c1 + ((capc * 4 + 255) & ~(size_t)255);
    if (cudaMallocAsync((void **)&base, o_c2 + capc * 4, st) != cudaSuccess) {
        cudaGetLastError();
        return GLASSO_ENOMEM;
    }
    struct Free {
        char *p;
        cudaStream_t st;
        ~Free() { cudaFreeAsync(p, st); }
    } guard{base, st};
    uint8_t *dmask = (uint8_t *)base;
    int32_t *dci = (int32_t *)(base + o_c1), *dcj = (int32_t *)(base + o_c2);
    int nmv = 0, ntr = 0;
    std::vector<uint8_t> mask((size_t)n);
    std::vector<int32_t> ci, cj, i1, i2;
    for (int64_t j0 = 0; j0 < n; j0 += block) {
        const int64_t j1 = std::min(j0 + block, n);
        i1.clear();
        i2.clear();
        for (int64_t i = 0; i < n; ++i) {
            mask[i] = i >= j0 && i < j1;
            (mask[i] ? i1 : i2).push_back((int32_t)i);
        }
        // F(A), log det A and W = A^{-1} at the current iterate
        double FA = 0.0;
        int info = 0;
        s = glasso_objective(ctx, S, A, n, lambda, &FA, &info);
        if (s != GLASSO_OK) return s;
        if (info != 0) return GLASSO_ENOTPD;
        CTX_CK(cudaMemcpyAsync(w.L, A, (size_t)(n * n) * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CTX_CK(potrf(w.L, n, w.xd, w.ldiag, w.sc, st));
        s = sync_ctx(ctx);
        if (s != GLASSO_OK) return s;
        const double ldA = w.sc_host->logdet;
        CTX_CK(inverse(w.L, n, w.W, w.T, w.U, st));
        // the block's candidates: pairs with a row or a column in I, from the
        // given candidates (in their order) or from all upper-triangle pairs (row-major)
        ci.clear();
        cj.clear();
        if (cand_i) {
            for (size_t p = 0; p < cand_i->size(); ++p) {
                const int32_t i = (*cand_i)[p], j = (*cand_j)[p];
                if (mask[i] || mask[j]) {
                    ci.push_back(i);
                    cj.push_back(j);
                }
            }
        } else {
            for (int64_t i = 0; i < n; ++i)
                for (int64_t j = i; j < n; ++j)
                    if (mask[i] || mask[j]) {
                        ci.push_back((int32_t)i);
                        cj.push_back((int32_t)j);
                    }
        }
        const int64_t nc = (int64_t)ci.size();
        if (nc == 0) continue;
        CTX_CK(cudaMemcpyAsync(dci, ci.data(), (size_t)nc * 4, cudaMemcpyHostToDevice, st));
        CTX_CK(cudaMemcpyAsync(dcj, cj.data(), (size_t)nc * 4, cudaMemcpyHostToDevice, st));
        CTX_CK(cudaMemcpyAsync(dmask, mask.data(), (size_t)n, cudaMemcpyHostToDevice, st));
        CTX_CK(scan_cand(S, w.W, A, n, lambda, dci, dcj, nullptr, 0, nc, w, w.pi, w.pj, nullptr, w.sc, st));
        s = sync_ctx(ctx);
        if (s != GLASSO_OK) return s;
        const int64_t np = w.sc_host->count;
        if (np == 0) continue;
        CTX_CK(pair_prep(S, w.W, A, n, lambda, w.pi, w.pj, np, w.p_inva, w.p_g, w.p_a, w.p_s, st));
        CTX_CK(cudaMemsetAsync(w.U, 0, (size_t)(n * n) * sizeof(double), st));
        CTX_CK(cudaMemsetAsync(w.D, 0, np * sizeof(double), st));
        if (inner == GLASSO_INNER_PCD_CG) {
            int its = 0;
            const cudaError_t pe = pcd(w.W, n, lambda, w.pi, w.pj, np, w.p_inva, w.p_g, w.p_a, kPcdIters, 1,
                                       kPcdRtol, w.D, w.U, w.T, false, w, st, &its);
            if (pe == cudaErrorLaunchTimeout) {
                ctx->last_error = "PCD-CG: a bounded grid-barrier wait expired";
                return GLASSO_ETIMEOUT;
            }
            CTX_CK(pe);
        } else {
            CTX_CK(cd_sweeps(w.W, n, lambda, w.pi, w.pj, np, w.p_inva, w.p_g, w.p_a, nsweeps, w.D, w.U, w, st));
        }
        CTX_CK(ls_delta(w.p_g, w.p_a, w.p_s, w.D, w.pi, w.pj, np, lambda, w, w.sc, st));
        s = sync_ctx(ctx);
        if (s != GLASSO_OK) return s;
        if (w.sc_host->bar_err) {
            ctx->last_error = "CD sweep: a bounded grid-barrier wait expired";
            return GLASSO_ETIMEOUT;
        }
        if (!w.sc_host->moved) continue;
        ++nmv;
        const double delta = w.sc_host->delta, trSD = w.sc_host->trSD;
        const double epsF = 1e-12 * std::max(fabs(FA), (double)n);
        double alpha = 1.0, a_acc = 0.0, prevF = INFINITY, prevA = 0.0;
        bool ok = false;
        for (int t = 0; t < 30 && !ok; ++t, alpha *= 0.5) {
            double ldT = 0.0;
            int code = 0;
            s = bcd_logdet_dev(ctx, A, n, w.pi, w.pj, np, w.D, dmask, i1, i2, alpha, &ldT, &code);
            if (s != GLASSO_OK) return s;
            CTX_CK(ls_dl1(w.p_a, w.D, w.pi, w.pj, np, alpha, w, w.sc, st));
            s = sync_ctx(ctx);
            if (s != GLASSO_OK) return s;
            ++ntr;
            const double Ft =
                code == 0 ? FA - (ldT - ldA) + alpha * trSD + lambda * w.sc_host->dl1 : INFINITY;
            if (rule == 0) {
                if (Ft <= FA + 1e-4 * alpha * delta + epsF) {
                    ok = true;
                    a_acc = alpha;
                }
            } else {
                if (prevF < INFINITY && prevF <= FA + epsF && Ft >= prevF) {
                    ok = true;
                    a_acc = prevA;
                }
                prevF = Ft;
                prevA = alpha;
            }
        }
        if (!ok && rule == 1 && prevF <= FA + epsF) {
            ok = true;  // the samples fell to the last one
            a_acc = prevA;
        }
        if (!ok) {
            if (moved) *moved = nmv;
            if (trials) *trials = ntr;
            return GLASSO_ELINESEARCH;
        }
        CTX_CK(ls_apply(A, n, w.pi, w.pj, w.p_a, w.D, np, a_acc, st));
        CTX_CK(cudaStreamSynchronize(st));
    }
    if (F_out) {
        int info = 0;
        s = glasso_objective(ctx, S, A, n, lambda, F_out, &info);
        if (s != GLASSO_OK) return s;
        if (info != 0) return GLASSO_ENOTPD;
    }
    if (moved) *moved = nmv;
    if (trials) *trials = ntr;
    return GLASSO_OK;
}

glasso_status glasso_bcd_iteration(glasso_ctx *ctx, const double *S, double *A, int64_t n, double lambda,
                                   int64_t block, int inner, int nsweeps, int rule, double *F_out,
                                   int *moved, int *trials) {
    if (!ctx || !S || !A || n < 1 || n > 46340 || !finite_pos(lambda) || block < 0 ||
        (inner != GLASSO_INNER_CD && inner != GLASSO_INNER_PCD_CG) || (rule != 0 && rule != 1) ||
        (inner == GLASSO_INNER_CD && nsweeps < 1))
        return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    return bcd_iteration_impl(ctx, S, A, n, lambda, block, inner, nsweeps, rule, nullptr, nullptr, F_out, moved,
                              trials);
}

// ML-BCD: Algorithm 1's control (hierarchy of Section 7, the Section 8 KKT
// stop) on the host, each relaxation one BCD-IC iteration on C_l.
glasso_status glasso_solve_bcd(glasso_ctx *ctx, const double *S, int64_t n, double lambda, double tol,
                               int max_cycles, int64_t block, int inner, int rule, int one_level, double *A,
                               glasso_info *info) {
    if (!ctx || !S || !A || n < 1 || n > 46340 || !finite_pos(lambda) || !(tol >= 0.0) || block < 0 ||
        (inner != GLASSO_INNER_CD && inner != GLASSO_INNER_PCD_CG) || (rule != 0 && rule != 1))
        return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    Work &w = ctx->w;
    cudaStream_t st = ctx->stream;
    glasso_status s = work_ensure(w, n, st, ctx->last_error);
    if (s != GLASSO_OK) return s;
    DevScalars *sc = w.sc, *h = w.sc_host;
    const int mc = max_cycles > 0 ? max_cycles : 200;
    const auto t0 = std::chrono::steady_clock::now();
    glasso_status status = GLASSO_EMAXITER;
    int cycles = 0, relax = 0, lstrials = 0;
    double relkkt = INFINITY, maxkkt = INFINITY, F = 0.0, logdet = 0.0;
    long long nnz = 0, max_nnz = 0;
    bool fresh = false;
    int64_t nf = 0;
    std::vector<int32_t> hfi, hfj, ci, cj;
    std::vector<uint8_t> htag;
    CTX_CK(cudaMemsetAsync(sc, 0, sizeof(DevScalars), st));
    CTX_CK(init_diag(S, n, lambda, A, sc, st));
    CTX_CK(cudaMemcpyAsync(w.L, A, (size_t)(n * n) * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CTX_CK(potrf(w.L, n, w.xd, w.ldiag, sc, st));
    s = sync_ctx(ctx);
    if (s != GLASSO_OK) return s;
    if (h->err || h->info != 0) return GLASSO_ENOTPD;
    CTX_CK(inverse(w.L, n, w.W, w.T, w.U, st));
    // initial free set (Section 7 footnote) with |G| on it
    CTX_CK(scan_full(S, w.W, A, n, lambda, 1, w, w.fi, w.fj, w.fabsg, sc, st));
    s = sync_ctx(ctx);
    if (s != GLASSO_OK) return s;
    nf = h->count;
    for (int k = 0; k < mc; ++k) {
        cycles = k + 1;
        const int nsweeps = std::min(1 + k / 3, 10);
        int Lv = 0;
        if (!one_level) {
            CTX_CK(support_flags(A, n, w.fi, w.fj, nf, w.fsupp, st));
            CTX_CK(hierarchy(w.fabsg, w.fsupp, nf, w.ftag, sc, st));
            s = sync_ctx(ctx);
            if (s != GLASSO_OK) return s;
            Lv = h->levels;
        }
        if (Lv > 0) {
            hfi.resize((size_t)nf);
            hfj.resize((size_t)nf);
            htag.resize((size_t)nf);
            CTX_CK(cudaMemcpyAsync(hfi.data(), w.fi, (size_t)nf * 4, cudaMemcpyDeviceToHost, st));
            CTX_CK(cudaMemcpyAsync(hfj.data(), w.fj, (size_t)nf * 4, cudaMemcpyDeviceToHost, st));
            CTX_CK(cudaMemcpyAsync(htag.data(), w.ftag, (size_t)nf, cudaMemcpyDeviceToHost, st));
            CTX_CK(cudaStreamSynchronize(st));
        }
        for (int l = Lv; l >= 0; --l) {
            fresh = false;
            const std::vector<int32_t> *pci = nullptr, *pcj = nullptr;
            if (l == 0) {
                // the fine free set at the current iterate, the KKT stop
                CTX_CK(cudaMemcpyAsync(w.L, A, (size_t)(n * n) * sizeof(double), cudaMemcpyDeviceToDevice, st));
                CTX_CK(potrf(w.L, n, w.xd, w.ldiag, sc, st));
                s = sync_ctx(ctx);
                if (s != GLASSO_OK) return s;
                if (h->info != 0) return GLASSO_ENOTPD;
                logdet = h->logdet;
                CTX_CK(inverse(w.L, n, w.W, w.T, w.U, st));
                CTX_CK(scan_full(S, w.W, A, n, lambda, 0, w, w.pi, w.pj, w.pabsg, sc, st));
                s = sync_ctx(ctx);
                if (s != GLASSO_OK) return s;
                const int64_t np = h->count;
                relkkt = h->kkt_sum / h->l1;
                maxkkt = h->kkt_max;
                nnz = h->nnz;
                max_nnz = std::max(max_nnz, nnz);
                F = -logdet + h->trSA + lambda * h->l1;
                CTX_CK(cudaMemcpyAsync(w.fi, w.pi, np * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
                CTX_CK(cudaMemcpyAsync(w.fj, w.pj, np * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
                CTX_CK(cudaMemcpyAsync(w.fabsg, w.pabsg, np * sizeof(double), cudaMemcpyDeviceToDevice, st));
                nf = np;
                fresh = true;
                if (relkkt <= tol) {
                    status = GLASSO_OK;
                    goto done;
                }
            } else {
                ci.clear();
                cj.clear();
                for (size_t p = 0; p < hfi.size(); ++p)
                    if (htag[p] >= l) {
                        ci.push_back(hfi[p]);
                        cj.push_back(hfj[p]);
                    }
                pci = &ci;
                pcj = &cj;
            }
            int tr = 0, mv = 0;
            s = bcd_iteration_impl(ctx, S, A, n, lambda, block, inner, nsweeps, rule, pci, pcj, nullptr, &mv, &tr);
            lstrials += tr;
            if (s == GLASSO_ELINESEARCH) {
                status = s;
                goto done;
            }
            if (s != GLASSO_OK) return s;
            if (mv) fresh = false;
            ++relax;
        }
    }
done:
    if (!fresh) {
        CTX_CK(cudaMemcpyAsync(w.L, A, (size_t)(n * n) * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CTX_CK(potrf(w.L, n, w.xd, w.ldiag, sc, st));
        s = sync_ctx(ctx);
        if (s != GLASSO_OK) return s;
        if (h->info == 0) {
            logdet = h->logdet;
            CTX_CK(inverse(w.L, n, w.W, w.T, w.U, st));
            CTX_CK(scan_full(S, w.W, A, n, lambda, 0, w, w.pi, w.pj, w.pabsg, sc, st));
            s = sync_ctx(ctx);
            if (s != GLASSO_OK) return s;
            relkkt = h->kkt_sum / h->l1;
            maxkkt = h->kkt_max;
            nnz = h->nnz;
            F = -logdet + h->trSA + lambda * h->l1;
        }
    }
    max_nnz = std::max(max_nnz, nnz);
    if (info) {
        memset(info, 0, sizeof(glasso_info));
        info->status = status;
        info->cycles = cycles;
        info->relaxations = relax;
        info->ls_trials = lstrials;
        info->objective = F;
        info->rel_kkt = relkkt;
        info->max_kkt = maxkkt;
        info->logdet = logdet;
        info->nnz = nnz;
        info->max_nnz = max_nnz;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return status;
}

glasso_status glasso_cholinv_mixed(glasso_ctx *ctx, const double *A, int64_t n, double *W, int *info,
                                   double *logdet) {
    if (!ctx || !A || !W || n < 1) return GLASSO_EINVAL;
    if (ctx->precision != GLASSO_MIXED) return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    glasso_status s = work_ensure(ctx->w, n, ctx->stream, ctx->last_error);
    if (s != GLASSO_OK) return s;
    s = work_ensure_mixed(ctx->w, n, ctx->stream, ctx->last_error);
    if (s != GLASSO_OK) return s;
    Work &w = ctx->w;
    const int64_t ldf = tc_pad(n);
    float *FA = w.fa, *FX = FA + n * ldf, *FXt = FX + n * ldf, *FZ = FXt + n * ldf;
    float *W32 = (float *)w.L;
    Prof *prof = (Prof *)ctx->prof;
    Solver sv{w, ctx->stream, ctx->last_error, prof};
    cudaEvent_t eb;
    CTX_CK(cudaMemsetAsync(w.sc, 0, sizeof(DevScalars), ctx->stream));
    CTX_CK(trial32(A, FA, n, ldf, nullptr, nullptr, nullptr, nullptr, 0, 0.0, ctx->stream));
    sv.mark_begin(4, eb);
    CTX_CK(ensure_side(w));
    CTX_CK(cholinv_tc(FA, n, ldf, FX, FXt, FZ, w.ldiag, w.sc, ctx->stream, w.side, w.ev_a, w.ev_b,
                            w.dbg_dag_tiles, w.dag_share));
    sv.mark_end(4, eb, 2.0 * (double)n * n * n / 3.0);
    s = sync_ctx(ctx);
    if (s != GLASSO_OK) return s;
    if (w.sc_host->tc_err) {
        ctx->last_error = "tensor-core factorisation: a bounded wait expired";
        return GLASSO_ETIMEOUT;
    }
    if (info) *info = w.sc_host->info;
    if (logdet) *logdet = w.sc_host->logdet;
    if (w.sc_host->info == 0) {
        sv.mark_begin(1, eb);
        CTX_CK(lauum_tc(FXt, n, ldf, W32, n, w.sc, ctx->stream));
        CTX_CK(to_f64(W32, W, n * n, ctx->stream));
        sv.mark_end(1, eb, (double)n * n * n / 3.0);
        s = sync_ctx(ctx);
        if (s != GLASSO_OK) return s;
        if (w.sc_host->tc_err) {
            ctx->last_error = "tensor-core GEMM: a bounded wait expired";
            return GLASSO_ETIMEOUT;
        }
    }
    if (prof) prof_collect(prof);
    return GLASSO_OK;
}

glasso_status glasso_free_set(glasso_ctx *ctx, const double *S, const double *W, const double *A,
                              int64_t n, double lambda, const int32_t *cand_i,
                              const int32_t *cand_j, int64_t ncand, int32_t *out_i,
                              int32_t *out_j, double *absg, int64_t *count, double *rel_kkt,
                              double *max_kkt) {
    if (!ctx || !S || !W || !A || n < 1 || !finite_pos(lambda) || !out_i || !out_j || !count)
        return GLASSO_EINVAL;
    if (cand_i && (!cand_j || ncand < 0)) return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    glasso_status s = work_ensure(ctx->w, n, ctx->stream, ctx->last_error);
    if (s != GLASSO_OK) return s;
    if (cand_i && ncand > ctx->w.cap_pairs) return GLASSO_EINVAL;
    Work &w = ctx->w;
    if (!cand_i) {
        CTX_CK(scan_full(S, W, A, n, lambda, 0, w, out_i, out_j, absg, w.sc, ctx->stream));
    } else {
        CTX_CK(scan_cand(S, W, A, n, lambda, cand_i, cand_j, nullptr, 0, ncand, w, out_i, out_j,
                         absg, w.sc, ctx->stream));
    }
    s = sync_ctx(ctx);
    if (s != GLASSO_OK) return s;
    *count = w.sc_host->count;
    if (!cand_i) {
        if (rel_kkt) *rel_kkt = w.sc_host->kkt_sum / w.sc_host->l1;
        if (max_kkt) *max_kkt = w.sc_host->kkt_max;
    }
    return GLASSO_OK;
}

glasso_status glasso_hierarchy(glasso_ctx *ctx, const double *absg, const uint8_t *insupp,
                               int64_t nf, uint8_t *tag, int *levels) {
    if (!ctx || nf < 0 || (nf > 0 && (!absg || !insupp || !tag)) || !levels) return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    glasso_status s = work_ensure(ctx->w, 1, ctx->stream, ctx->last_error);
    if (s != GLASSO_OK) return s;
    CTX_CK(hierarchy(absg, insupp, nf, tag, ctx->w.sc, ctx->stream));
    s = sync_ctx(ctx);
    if (s != GLASSO_OK) return s;
    *levels = ctx->w.sc_host->levels;
    return GLASSO_OK;
}

glasso_status glasso_cd_sweeps(glasso_ctx *ctx, const double *S, const double *W, const double *A,
                               int64_t n, double lambda, const int32_t *pi, const int32_t *pj,
                               int64_t np, int nsweeps, double *D, double *U) {
    if (!ctx || !S || !W || !A || n < 1 || !finite_pos(lambda) || np < 0 || nsweeps < 0 ||
        (np > 0 && (!pi || !pj || !D || !U)))
        return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    glasso_status s = work_ensure(ctx->w, n, ctx->stream, ctx->last_error);
    if (s != GLASSO_OK) return s;
    if (np > ctx->w.cap_pairs) return GLASSO_EINVAL;
    Work &w = ctx->w;
    Prof *prof = (Prof *)ctx->prof;
    Solver sv{w, ctx->stream, ctx->last_error, prof};
    CTX_CK(pair_prep(S, W, A, n, lambda, pi, pj, np, w.p_inva, w.p_g, w.p_a, w.p_s, ctx->stream));
    cudaEvent_t eb;
    sv.mark_begin(3, eb);
    if (ctx->precision == GLASSO_MIXED) {
        // the mixed solve's sweep: W and U in FP32 (FP32 resolution chain,
        // FP64 increments), U converted back; scratch in the FP64 buffers
        const int64_t nn = n * n;
        float *W32 = reinterpret_cast<float *>(w.L), *U32 = reinterpret_cast<float *>(w.W);
        float *U2 = reinterpret_cast<float *>(w.T);
        CTX_CK(to_f32(W, W32, nn, ctx->stream));
        CTX_CK(to_f32(U, U32, nn, ctx->stream));
        CTX_CK(cd_sweeps32(W32, n, lambda, pi, pj, np, w.p_inva, w.p_g, w.p_a, nsweeps, D, U32, w, false,
                           ctx->stream, U2));
        CTX_CK(to_f64(U32, U, nn, ctx->stream));
    } else {
        CTX_CK(cd_sweeps(W, n, lambda, pi, pj, np, w.p_inva, w.p_g, w.p_a, nsweeps, D, U, w, ctx->stream));
    }
    sv.mark_end(3, eb, (double)nsweeps * (double)np * 6.0 * (double)n * 8.0);
    s = sync_ctx(ctx);
    if (prof) prof_collect(prof);
    if (s != GLASSO_OK) return s;
    if (w.sc_host->bar_err) {
        ctx->last_error = "CD sweep: a bounded grid-barrier wait expired";
        return GLASSO_ETIMEOUT;
    }
    return GLASSO_OK;
}

glasso_status glasso_pcd(glasso_ctx *ctx, const double *S, const double *W, const double *A, int64_t n,
                         double lambda, const int32_t *pi, const int32_t *pj, int64_t np, int iters,
                         int cg, double rtol, double *D, double *U, int *iters_done) {
    if (!ctx || !S || !W || !A || !U || n < 1 || !finite_pos(lambda) || np < 0 || iters < 0 ||
        !(rtol >= 0.0) || (np > 0 && (!pi || !pj || !D)))
        return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    glasso_status s = work_ensure(ctx->w, n, ctx->stream, ctx->last_error);
    if (s != GLASSO_OK) return s;
    if (np > ctx->w.cap_pairs) return GLASSO_EINVAL;
    Work &w = ctx->w;
    cudaStream_t st = ctx->stream;
    int its = 0;
    CTX_CK(pair_prep(S, W, A, n, lambda, pi, pj, np, w.p_inva, w.p_g, w.p_a, w.p_s, st));
    if (ctx->precision == GLASSO_MIXED) {
        // the mixed solve's arithmetic: the products with W in FP32
        const int64_t nn = n * n;
        float *W32 = reinterpret_cast<float *>(w.L), *U32 = reinterpret_cast<float *>(w.W);
        float *Vt = reinterpret_cast<float *>(w.T);
        CTX_CK(to_f32(W, W32, nn, st));
        const cudaError_t pe = pcd32(W32, n, lambda, pi, pj, np, w.p_inva, w.p_g, w.p_a, iters, cg, rtol, D,
                                     U32, Vt, true, w, st, &its);
        if (pe == cudaErrorLaunchTimeout) {
            ctx->last_error = "PCD-CG: a bounded grid-barrier wait expired";
            return GLASSO_ETIMEOUT;
        }
        CTX_CK(pe);
        CTX_CK(to_f64(U32, U, nn, st));
    } else {
        const cudaError_t pe = pcd(W, n, lambda, pi, pj, np, w.p_inva, w.p_g, w.p_a, iters, cg, rtol, D, U, w.T,
                                   true, w, st, &its);
        if (pe == cudaErrorLaunchTimeout) {
            ctx->last_error = "PCD-CG: a bounded grid-barrier wait expired";
            return GLASSO_ETIMEOUT;
        }
        CTX_CK(pe);
    }
    s = sync_ctx(ctx);
    if (s != GLASSO_OK) return s;
    if (iters_done) *iters_done = its;
    return GLASSO_OK;
}

glasso_status glasso_line_search(glasso_ctx *ctx, const double *S, const double *W, double *A,
                                 int64_t n, double lambda, const int32_t *pi, const int32_t *pj,
                                 int64_t np, const double *D, double F_A, double sigma,
                                 int max_trials, double *F_new, double *alpha, int *trials) {
    if (!ctx || !S || !W || !A || n < 1 || !finite_pos(lambda) || np < 0 || max_trials < 1 ||
        (np > 0 && (!pi || !pj || !D)))
        return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    glasso_status s = work_ensure(ctx->w, n, ctx->stream, ctx->last_error);
    if (s != GLASSO_OK) return s;
    if (np > ctx->w.cap_pairs) return GLASSO_EINVAL;
    Work &w = ctx->w;
    cudaStream_t st = ctx->stream;
    CTX_CK(pair_prep(S, W, A, n, lambda, pi, pj, np, w.p_inva, w.p_g, w.p_a, w.p_s, st));
    CTX_CK(ls_delta(w.p_g, w.p_a, w.p_s, D, pi, pj, np, lambda, w, w.sc, st));
    s = sync_ctx(ctx);
    if (s != GLASSO_OK) return s;
    const double delta = w.sc_host->delta, trSD = w.sc_host->trSD;
    // tr(SA) and ||A||_1 of the current iterate from F_A's definition are not
    // needed: F(A + alpha Delta) - F(A) only involves the pairs.
    double a = 1.0;
    const double epsF = 1e-12 * std::max(fabs(F_A), (double)n);
    double ldA = 0.0;
    // log det A itself (to express F(A + alpha Delta) relative to F_A)
    CTX_CK(cudaMemcpyAsync(w.T, A, (size_t)(n * n) * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CTX_CK(potrf(w.T, n, w.xd, w.ldiag, w.sc, st));
    s = sync_ctx(ctx);
    if (s != GLASSO_OK) return s;
    if (w.sc_host->info != 0) return GLASSO_EINVAL;
    ldA = w.sc_host->logdet;
    for (int t = 0; t < max_trials; ++t) {
        CTX_CK(ls_build_trial(A, w.T, n, pi, pj, w.p_a, D, np, a, st));
        CTX_CK(potrf(w.T, n, w.xd, w.ldiag, w.sc, st));
        CTX_CK(ls_dl1(w.p_a, D, pi, pj, np, a, w, w.sc, st));
        s = sync_ctx(ctx);
        if (s != GLASSO_OK) return s;
        if (w.sc_host->info == 0 && !w.dbg_ls_reject) {
            const double FT = F_A - (w.sc_host->logdet - ldA) + a * trSD + lambda * w.sc_host->dl1;
            if (FT <= F_A + sigma * a * delta + epsF) {
                CTX_CK(ls_apply(A, n, pi, pj, w.p_a, D, np, a, st));
                CTX_CK(cudaStreamSynchronize(st));
                if (F_new) *F_new = FT;
                if (alpha) *alpha = a;
                if (trials) *trials = t + 1;
                return GLASSO_OK;
            }
        }
        a *= 0.5;
    }
    if (trials) *trials = max_trials;
    if (alpha) *alpha = 0.0;
    return GLASSO_ELINESEARCH;
}

glasso_status glasso_components(glasso_ctx *ctx, const double *S, int64_t n, double lambda,
                                int32_t *comp, int64_t *ncomp) {
    if (!ctx || !S || !comp || n < 1 || n > 46340 || !finite_pos(lambda)) return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    Work &w = ctx->w;
    cudaStream_t st = ctx->stream;
    glasso_status s = work_ensure(w, 1, st, ctx->last_error);  // the device scalars
    if (s == GLASSO_OK) s = work_ensure_labels(w, n, st, ctx->last_error);
    if (s != GLASSO_OK) return s;
    CTX_CK(cudaMemsetAsync(&w.sc->cc_err, 0, sizeof(int), st));
    CTX_CK(components(S, n, lambda, w.cc_parent, comp, w.cc_size, &w.sc->cc_err, st));
    std::vector<int> size;
    if (ncomp) {
        size.resize((size_t)n);
        CTX_CK(cudaMemcpyAsync(size.data(), w.cc_size, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    s = sync_ctx(ctx);
    if (s != GLASSO_OK) return s;
    if (w.sc_host->cc_err) {
        ctx->last_error = "component labelling: a retry bound was exceeded";
        return GLASSO_ECUDA;
    }
    if (ncomp) *ncomp = (int64_t)std::count_if(size.begin(), size.end(), [](int c) { return c > 0; });
    return GLASSO_OK;
}

glasso_status glasso_objective(glasso_ctx *ctx, const double *S, const double *A, int64_t n,
                               double lambda, double *F, int *info) {
    if (!ctx || !S || !A || n < 1 || !finite_pos(lambda) || !F || !info) return GLASSO_EINVAL;
    cudaSetDevice(ctx->device);
    glasso_status s = work_ensure(ctx->w, n, ctx->stream, ctx->last_error);
    if (s != GLASSO_OK) return s;
    Work &w = ctx->w;
    cudaStream_t st = ctx->stream;
    CTX_CK(cudaMemcpyAsync(w.T, A, (size_t)(n * n) * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CTX_CK(potrf(w.T, n, w.xd, w.ldiag, w.sc, st));
    // tr(SA) and ||A||_1 come with a scan whose W is S itself (G = 0): only the
    // trace and l1 sums are read from it.
    CTX_CK(scan_full(S, S, A, n, lambda, 0, w, w.pi, w.pj, nullptr, w.sc, st));
    s = sync_ctx(ctx);
    if (s != GLASSO_OK) return s;
    *info = w.sc_host->info;
    *F = -w.sc_host->logdet + w.sc_host->trSA + lambda * w.sc_host->l1;
    return GLASSO_OK;
}

}  // extern "C"
