/*
 * FP64 CPU oracle for the multilevel proximal-Newton solver of the
 * l1-regularised log-det problem (Treister, Turek, Yavneh, arXiv 1607.00315).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference against which the CUDA path is checked.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or helper with the CUDA library, and the CUDA library
 * never calls it.
 *
 * Problem (Section 5, eq. MLE_l1_prior):
 *     min_{A > 0}  F(A) = -log det A + tr(S A) + lambda * sum_ij |A_ij|
 * The diagonal is penalised.  The minimiser is unique.
 *
 * All matrices are dense, row-major, n x n, double precision.  Pair lists hold
 * upper-triangle index pairs (i <= j) in row-major order (i ascending, then j
 * ascending); a pair (i, j) stands for both A_ij and A_ji.
 *
 * Functions: a1-a8 (the dense ML-cycle: S, Cholesky, inverse, free set and
 * KKT residual, hierarchy, CD sweeps, PCD / PCD-CG, line search, solve),
 * continuation and screening, and NEXT-4: BCD-IC (Section 6, Algorithm 2) with
 * its Schur-complement log det and ML-BCD (the ML-cycle over BCD-IC).
 *
 * Readings of points the paper leaves open are marked READING.
 * Parity pins: every function here is pinned by the CPU test suite against
 * closed forms, library routines, brute force on tiny inputs or the paper's
 * optimality conditions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ENOTPD 3
#define ORC_ELINESEARCH 4
#define ORC_EMAXITER 5
#define ORC_EINVAL 1

static double sgn(double x) { return (x > 0.0) - (x < 0.0); }

/* Soft shrinkage S_t(x) = sign(x) * max(0, |x| - t), eq. shrinkage (Section 2). */
static double soft(double x, double t) {
    double ax = fabs(x) - t;
    return ax > 0.0 ? sgn(x) * ax : 0.0;
}

/* ---------------------------------------------------------------------- */
/* a1. Empirical covariance, eq. cov_estimate (Section 5):
 *     S = (1/m) sum_k (y_k - mu)(y_k - mu)^T,  mu = mean of the samples when
 *     `center` is set, else zero.  X is m x n (one sample per row).         */
void orc_form_S(const double *X, int64_t m, int64_t n, int center, double *S) {
    double *mu = (double *)calloc((size_t)n, sizeof(double));
    if (center) {
        for (int64_t k = 0; k < m; ++k)
            for (int64_t i = 0; i < n; ++i) mu[i] += X[k * n + i];
        for (int64_t i = 0; i < n; ++i) mu[i] /= (double)m;
    }
    /* the sum of outer products of eq. cov_estimate, one sample at a time */
    memset(S, 0, (size_t)(n * n) * sizeof(double));
    for (int64_t k = 0; k < m; ++k) {
        const double *y = X + k * n;
        for (int64_t i = 0; i < n; ++i) {
            double yi = y[i] - mu[i];
            for (int64_t j = 0; j <= i; ++j) S[i * n + j] += yi * (y[j] - mu[j]);
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j <= i; ++j) {
            S[i * n + j] /= (double)m;
            S[j * n + i] = S[i * n + j];
        }
    free(mu);
}

/* ---------------------------------------------------------------------- */
/* a2. Cholesky factorisation A = L L^T (textbook column-by-column form).
 * Returns 0 on success or k+1 when the k-th pivot is not positive (A is not
 * positive definite; the line-search PD test of Section 6.1.2).  L is lower
 * triangular with zeros above the diagonal.                                */
int orc_cholesky(const double *A, int64_t n, double *L) {
    memset(L, 0, (size_t)(n * n) * sizeof(double));
    for (int64_t j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int64_t k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        if (!(d > 0.0)) return (int)(j + 1);
        double ljj = sqrt(d);
        L[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int64_t k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = s / ljj;
        }
    }
    return 0;
}

/* log det A = 2 sum_i log L_ii for A = L L^T. */
double orc_logdet_from_chol(const double *L, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += log(L[i * n + i]);
    return 2.0 * s;
}

/* a3. W = A^{-1} = L^{-T} L^{-1} from the Cholesky factor (eq. gradHes needs
 * A^{-1}).  X = L^{-1} is found column by column by forward substitution
 * (L x_k = e_k, x_k zero above k); the columns are stored as rows of
 * Y = X^T so that W_ij = sum_t X_ti X_tj = sum_t Y_it Y_jt runs along rows. */
void orc_inverse_from_chol(const double *L, int64_t n, double *W) {
    double *Y = (double *)calloc((size_t)(n * n), sizeof(double));
    for (int64_t k = 0; k < n; ++k) {
        double *y = Y + k * n; /* column k of L^{-1} */
        for (int64_t i = k; i < n; ++i) {
            double s = (i == k) ? 1.0 : 0.0;
            for (int64_t t = k; t < i; ++t) s -= L[i * n + t] * y[t];
            y[i] = s / L[i * n + i];
        }
    }
    /* W = X^T X: entry (i, j) sums over t >= max(i, j) where both are nonzero */
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j <= i; ++j) {
            double s = 0.0;
            for (int64_t t = i; t < n; ++t) s += Y[i * n + t] * Y[j * n + t];
            W[i * n + j] = s;
            W[j * n + i] = s;
        }
    free(Y);
}

/* tr(S A) and ||A||_1 = sum_ij |A_ij| (eq. MLE_l1_prior). */
static void trace_and_l1(const double *S, const double *A, int64_t n, double *tr, double *l1) {
    double t = 0.0, a = 0.0;
    for (int64_t i = 0; i < n * n; ++i) {
        t += S[i] * A[i];
        a += fabs(A[i]);
    }
    *tr = t;
    *l1 = a;
}

/* F(A) = -log det A + tr(SA) + lambda ||A||_1 (eq. MLE_l1_prior).
 * Returns 0, or the Cholesky info when A is not positive definite.         */
int orc_objective(const double *S, const double *A, int64_t n, double lam, double *F) {
    double *L = (double *)malloc((size_t)(n * n) * sizeof(double));
    int info = orc_cholesky(A, n, L);
    if (info == 0) {
        double tr, l1;
        trace_and_l1(S, A, n, &tr, &l1);
        *F = -orc_logdet_from_chol(L, n) + tr + lam * l1;
    }
    free(L);
    return info;
}

/* ---------------------------------------------------------------------- */
/* a4. Free set, eq. active_set (Section 5.2):
 *     F(A) = {(i,j) : A_ij != 0  or  |(S - A^{-1})_ij| > lambda}
 * restricted to a candidate set C_l (Section 7, eq. MLE_l1_prior_C).
 * When `cand` is NULL the candidates are all upper-triangle pairs.  The zero
 * test is exact (READING: the soft-shrinkage step yields exact zeros).
 * Writes the pairs in candidate order; returns their count.                */
int64_t orc_free_set(const double *S, const double *W, const double *A, int64_t n, double lam,
                     const int32_t *cand_i, const int32_t *cand_j, int64_t ncand,
                     int32_t *out_i, int32_t *out_j) {
    int64_t cnt = 0;
    if (cand_i == NULL) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = i; j < n; ++j) {
                double g = S[i * n + j] - W[i * n + j];
                if (A[i * n + j] != 0.0 || fabs(g) > lam) {
                    out_i[cnt] = (int32_t)i;
                    out_j[cnt] = (int32_t)j;
                    ++cnt;
                }
            }
    } else {
        for (int64_t p = 0; p < ncand; ++p) {
            int64_t i = cand_i[p], j = cand_j[p];
            double g = S[i * n + j] - W[i * n + j];
            if (A[i * n + j] != 0.0 || fabs(g) > lam) {
                out_i[cnt] = (int32_t)i;
                out_j[cnt] = (int32_t)j;
                ++cnt;
            }
        }
    }
    return cnt;
}

/* Relative KKT residual (Section 8 stopping rule, with the subdifferential of
 * eq. subgradient1): the minimum-norm subgradient
 *     g_ij = G_ij + lambda sign(A_ij)                   if A_ij != 0
 *     g_ij = sign(G_ij) max(|G_ij| - lambda, 0)         if A_ij == 0
 * with G = S - W, summed in absolute value over all (i, j) and divided by
 * ||A||_1.  Also returns max_ij |g_ij|.                                    */
double orc_rel_kkt(const double *S, const double *W, const double *A, int64_t n, double lam,
                   double *maxabs) {
    double num = 0.0, den = 0.0, mx = 0.0;
    for (int64_t i = 0; i < n * n; ++i) {
        double g = S[i] - W[i];
        double r = (A[i] != 0.0) ? g + lam * sgn(A[i]) : soft(g, lam);
        num += fabs(r);
        den += fabs(A[i]);
        if (fabs(r) > mx) mx = fabs(r);
    }
    if (maxabs) *maxabs = mx;
    return num / den;
}

/* ---------------------------------------------------------------------- */
/* a5. Multilevel hierarchy (Section 3.2 and Section 7):
 * Given the previous fine-level free set F_k (nf pairs), the absolute
 * gradient |G| on those pairs and a flag telling which pairs are in
 * supp(A^(k)), build nested C_1 > ... > C_L = supp with
 *     |C_1| = max(ceil(|F_k| / 2), |supp|),
 *     |C_{l+1}| = max(ceil(|C_l| / 2), |supp|), stop when |C_l| = |supp|.
 * C_l = supp + the (|C_l| - |supp|) non-support pairs of largest |G|.
 * READING: ties in |G| are broken by list position (row-major pair order),
 * and when ceil(|F_k|/2) <= |supp| the hierarchy is C_1 = supp, L = 1.
 * Output: tag[p] = the coarsest level containing pair p (0 if p is only in
 * C_0), L via *levels.  Pairs outside F_k are in C_0 only.                  */
static const double *g_rank_key;
static int cmp_rank(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    double ka = g_rank_key[a], kb = g_rank_key[b];
    if (ka > kb) return -1; /* larger |G| first */
    if (ka < kb) return 1;
    return (a < b) ? -1 : (a > b); /* earlier pair first */
}

int orc_hierarchy(const double *absg, const uint8_t *insupp, int64_t nf, uint8_t *tag, int *levels) {
    int64_t ns = 0;
    for (int64_t p = 0; p < nf; ++p) ns += insupp[p] ? 1 : 0;
    int64_t sizes[64];
    int L = 1;
    int64_t s = (nf + 1) / 2;
    if (s < ns) s = ns;
    sizes[1] = s;
    while (sizes[L] > ns && L < 62) {
        int64_t nxt = (sizes[L] + 1) / 2;
        if (nxt < ns) nxt = ns;
        sizes[++L] = nxt;
    }
    *levels = L;
    int64_t nr = nf - ns;
    int64_t *order = (int64_t *)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(int64_t));
    int64_t q = 0;
    for (int64_t p = 0; p < nf; ++p)
        if (!insupp[p]) order[q++] = p;
    g_rank_key = absg;
    qsort(order, (size_t)nr, sizeof(int64_t), cmp_rank);
    for (int64_t p = 0; p < nf; ++p) tag[p] = insupp[p] ? (uint8_t)L : 0;
    for (int64_t r = 0; r < nr; ++r) {
        int t = 0;
        for (int l = 1; l <= L; ++l)
            if (r < sizes[l] - ns) t = l;
        tag[order[r]] = (uint8_t)t;
    }
    free(order);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* a6. Coordinate descent on the Newton LASSO, eq. Quad_MLE_l1_prior
 *     min_Delta tr(Delta G) + 1/2 tr(Delta W Delta W) + lambda ||A + Delta||_1
 * restricted to the given pairs (Section 5.2 free set, Section 7 restriction).
 * For an off-diagonal pair, Delta <- Delta + mu (e_i e_j^T + e_j e_i^T)
 * changes the model by 2 (b mu + a mu^2 / 2 + lambda |c + mu|) - 2 lambda |c|
 * with a = W_ij^2 + W_ii W_jj, b = G_ij + (W Delta W)_ij, c = A_ij + Delta_ij;
 * for a diagonal pair a = W_ii^2 and there is no factor 2.  In both cases
 * the 1-D minimiser (eq. 1d_l1) is mu = -c + S_{lambda/a}(c - b/a).
 * READING: the paper's printed closed form has the sign of (b -+ lambda)/a
 * reversed; the minimiser of a z^2/2 + b z + lambda |z| is -(b - lambda)/a
 * for b > lambda, which is what the formula above gives.
 * U = Delta W is kept up to date: (W Delta W)_ij = W_i,: . U_:,j and the
 * update adds mu W_j,: to row i of U and mu W_i,: to row j.  When the
 * shrinkage returns zero the new value A_ij + Delta_ij is set to exactly zero
 * (Delta_ij = -A_ij), so that the support test A_ij != 0 of eq. active_set
 * sees the zero the shrinkage prescribes rather than a rounding residue.
 * D holds Delta on the pair list (in/out); U is n x n (in/out).           */
void orc_cd_sweeps(const double *S, const double *W, const double *A, int64_t n, double lam,
                   const int32_t *pi, const int32_t *pj, int64_t np, int nsweeps,
                   double *D, double *U) {
    for (int sw = 0; sw < nsweeps; ++sw) {
        for (int64_t p = 0; p < np; ++p) {
            int64_t i = pi[p], j = pj[p];
            double wij = W[i * n + j];
            double a = (i == j) ? wij * wij : wij * wij + W[i * n + i] * W[j * n + j];
            double wdw = 0.0;
            for (int64_t k = 0; k < n; ++k) wdw += W[i * n + k] * U[k * n + j];
            double b = (S[i * n + j] - wij) + wdw;
            double c = A[i * n + j] + D[p];
            double z = soft(c - b / a, lam / a);
            double mu = -c + z;
            if (mu != 0.0) {
                /* a zero from the shrinkage is written exactly: A_ij + Delta_ij = 0 */
                if (z == 0.0) {
                    mu = -A[i * n + j] - D[p];
                    D[p] = -A[i * n + j];
                } else {
                    D[p] += mu;
                }
                for (int64_t k = 0; k < n; ++k) U[i * n + k] += mu * W[j * n + k];
                if (i != j)
                    for (int64_t k = 0; k < n; ++k) U[j * n + k] += mu * W[i * n + k];
            }
        }
    }
}

/* ---------------------------------------------------------------------- */
/* PCD and PCD-CG for the same Newton LASSO (the Jacobi-parallel alternative
 * to the CD sweep; the paper's inner solver of Section 6.3).
 *
 * Direction (Section 2, eq. IST_direction with D = diag of the Hessian, the
 * generalised parallel coordinate descent): every coordinate's own 1-D
 * minimiser at the current Delta, all taken at once,
 *     d_p = S_{lambda/a_p}(c_p - b_p/a_p) - c_p
 * with a, b, c as in the CD sweep above.
 * Step (eq. Line-search): the exact minimiser t >= 0 of the model along the
 * search direction.  Along Delta + t P the model changes by
 *     phi(t) = t g1 + t^2 g2 / 2 + lambda sum_p w_p (|c_p + t P_p| - |c_p|),
 *     g1 = sum_p w_p b_p P_p,  g2 = sum_p w_p P_p (W P W)_p,
 * w_p = 2 off the diagonal and 1 on it (a pair stands for two entries); phi
 * is a convex quadratic plus a piecewise-linear term, so its minimiser is
 * found by walking the kinks t = -c_p / P_p > 0 in increasing order.  When
 * the minimiser is a kink, the coordinates of that kink get exact zeros
 * (Delta_p = -A_p), as the CD sweep does for a zero of the shrinkage.
 * READING (zero snap): a coordinate whose own minimiser is zero (the
 * shrinkage returned 0, so d_p = -c_p) approaches zero only geometrically
 * when the step is shorter than its kink, and once its value lies below the
 * resolution of the update (Delta_p + t P_p rounds to Delta_p) it freezes at
 * a nonzero residue whose sign keeps pulling the other coordinates; plain PCD
 * then stalls.  Such a coordinate is set to its limit, the exact zero.
 * Acceleration by non-linear conjugate gradients (PCD-CG, Section 6.3).
 * READING (the paper defers the details to its references): the search
 * direction is P_k = d_k + beta_k P_{k-1} with the Polak-Ribiere-plus
 * coefficient beta_k = max(0, <d_k, d_k - d_{k-1}> / <d_{k-1}, d_{k-1}>) in
 * the w-weighted pair inner product; P_k = d_k when the directional
 * derivative phi'(0+) along P_k is not negative.  cg = 0: plain PCD.
 * Stops after `iters` iterations, when d = 0 (the LASSO minimiser), or, for
 * rtol > 0, once max|d| <= rtol * max|d| of the first iteration; on that
 * last stop, coordinates whose own minimiser is zero take their exact zero
 * (READING: the final shrinkage, below) (Section 8
 * stops its PCD-CG inner solves at relative precision 1e-4; READING: that
 * precision is measured by the PCD direction, zero exactly at the minimiser).
 * D holds Delta on the pair list (in/out); U = Delta W (n x n, in/out) is
 * updated with the exact increments.  Returns the iterations taken.         */

/* (W X W)_p on the pairs for the symmetric X given on the pairs: V = X W
 * (row updates), then the dot of row i of W with column j of V.  V: n x n. */
static void pair_wxw(const double *W, int64_t n, const int32_t *pi, const int32_t *pj,
                     int64_t np, const double *x, double *V, double *out) {
    memset(V, 0, (size_t)(n * n) * sizeof(double));
    for (int64_t p = 0; p < np; ++p) {
        const int64_t i = pi[p], j = pj[p];
        if (x[p] == 0.0) continue;
        for (int64_t k = 0; k < n; ++k) V[i * n + k] += x[p] * W[j * n + k];
        if (i != j)
            for (int64_t k = 0; k < n; ++k) V[j * n + k] += x[p] * W[i * n + k];
    }
    for (int64_t p = 0; p < np; ++p) {
        const int64_t i = pi[p], j = pj[p];
        double s = 0.0;
        for (int64_t k = 0; k < n; ++k) s += W[i * n + k] * V[k * n + j];
        out[p] = s;
    }
}

/* The PCD direction at the current Delta (D, U = Delta W): d_p as above and
 * b_p = G_p + (W Delta W)_p. */
void orc_pcd_direction(const double *S, const double *W, const double *A, int64_t n, double lam,
                       const int32_t *pi, const int32_t *pj, int64_t np, const double *D,
                       const double *U, double *d, double *b) {
    for (int64_t p = 0; p < np; ++p) {
        const int64_t i = pi[p], j = pj[p];
        const double wij = W[i * n + j];
        const double a = (i == j) ? wij * wij : wij * wij + W[i * n + i] * W[j * n + j];
        double wdw = 0.0;
        for (int64_t k = 0; k < n; ++k) wdw += W[i * n + k] * U[k * n + j];
        b[p] = (S[i * n + j] - wij) + wdw;
        const double c = A[i * n + j] + D[p];
        d[p] = soft(c - b[p] / a, lam / a) - c;
    }
}

typedef struct {
    double t;
    int64_t p;
} kink;

static int cmp_kink(const void *x, const void *y) {
    const kink *a = (const kink *)x, *b = (const kink *)y;
    if (a->t < b->t) return -1;
    if (a->t > b->t) return 1;
    return (a->p > b->p) - (a->p < b->p);
}

/* Exact minimiser t >= 0 of phi (above); *at_kink = the kink value when the
 * minimiser is one (else -1). */
static double exact_step(const double *c, const double *P, const double *w, int64_t np, double lam,
                         double g1, double g2, kink *ks, double *at_kink) {
    *at_kink = -1.0;
    double h = 0.0; /* lambda sum w P s, s = the sign just right of t */
    int64_t nk = 0;
    for (int64_t p = 0; p < np; ++p) {
        if (P[p] == 0.0) continue;
        const double s = c[p] != 0.0 ? sgn(c[p]) : sgn(P[p]);
        h += lam * w[p] * P[p] * s;
        if (c[p] != 0.0 && sgn(c[p]) != sgn(P[p])) {
            ks[nk].t = -c[p] / P[p];
            ks[nk].p = p;
            ++nk;
        }
    }
    if (!(g2 > 0.0) || g1 + h >= 0.0) return 0.0;
    qsort(ks, (size_t)nk, sizeof(kink), cmp_kink);
    int64_t k = 0;
    while (k < nk) {
        const double tk = ks[k].t;
        const double tstar = -(g1 + h) / g2;
        if (tstar <= tk) return tstar;
        /* crossing the kink(s) at tk: each sign flips from -sign(P) to sign(P) */
        double jump = 0.0;
        int64_t k2 = k;
        while (k2 < nk && ks[k2].t == tk) {
            jump += 2.0 * lam * w[ks[k2].p] * fabs(P[ks[k2].p]);
            ++k2;
        }
        if (g1 + g2 * tk + h + jump >= 0.0) {
            *at_kink = tk;
            return tk;
        }
        h += jump;
        k = k2;
    }
    return -(g1 + h) / g2;
}

int orc_pcd(const double *S, const double *W, const double *A, int64_t n, double lam,
            const int32_t *pi, const int32_t *pj, int64_t np, int iters, int cg, double rtol,
            double *D, double *U) {
    const size_t m = (size_t)(np > 0 ? np : 1);
    double *d = (double *)malloc(m * sizeof(double));
    double *dprev = (double *)malloc(m * sizeof(double));
    double *P = (double *)calloc(m, sizeof(double)); /* the previous direction: none yet */
    double *b = (double *)malloc(m * sizeof(double));
    double *c = (double *)malloc(m * sizeof(double));
    double *w = (double *)malloc(m * sizeof(double));
    double *wpw = (double *)malloc(m * sizeof(double));
    unsigned char *zt = (unsigned char *)malloc(m);
    kink *ks = (kink *)malloc(m * sizeof(kink));
    double *V = (double *)malloc((size_t)(n * n) * sizeof(double));
    int it = 0;
    double d0max = 0.0;
    for (int64_t p = 0; p < np; ++p) w[p] = pi[p] == pj[p] ? 1.0 : 2.0;
    for (; it < iters; ++it) {
        orc_pcd_direction(S, W, A, n, lam, pi, pj, np, D, U, d, b);
        double dmax = 0.0;
        for (int64_t p = 0; p < np; ++p) dmax = fmax(dmax, fabs(d[p]));
        if (dmax == 0.0) break;
        if (it == 0) d0max = dmax;
        else if (rtol > 0.0 && dmax <= rtol * d0max) {
            /* READING (final shrinkage): a coordinate whose own minimiser is
             * zero is left by the steps at a residue below the stopping
             * precision, on either side of zero; it takes its exact zero here,
             * as a coordinate-descent step on it would give */
            for (int64_t p = 0; p < np; ++p) {
                const int64_t i = pi[p], j = pj[p];
                const double cp = A[i * n + j] + D[p];
                if (cp == 0.0 || cp + d[p] != 0.0) continue;
                const double inc = -A[i * n + j] - D[p];
                D[p] = -A[i * n + j];
                for (int64_t k = 0; k < n; ++k) U[i * n + k] += inc * W[j * n + k];
                if (i != j)
                    for (int64_t k = 0; k < n; ++k) U[j * n + k] += inc * W[i * n + k];
            }
            break;
        }
        double beta = 0.0;
        if (cg && it > 0) {
            double num = 0.0, den = 0.0;
            for (int64_t p = 0; p < np; ++p) {
                num += w[p] * d[p] * (d[p] - dprev[p]);
                den += w[p] * dprev[p] * dprev[p];
            }
            beta = den > 0.0 ? fmax(0.0, num / den) : 0.0;
        }
        for (int64_t p = 0; p < np; ++p) {
            P[p] = d[p] + beta * P[p];
            c[p] = A[pi[p] * n + pj[p]] + D[p];
            zt[p] = c[p] + d[p] == 0.0; /* the coordinate's own minimiser is zero */
        }
        double g1 = 0.0;
        for (int64_t p = 0; p < np; ++p) g1 += w[p] * b[p] * P[p];
        if (beta != 0.0) {
            /* a descent direction or back to the PCD direction */
            double h = 0.0;
            for (int64_t p = 0; p < np; ++p)
                if (P[p] != 0.0) h += lam * w[p] * P[p] * (c[p] != 0.0 ? sgn(c[p]) : sgn(P[p]));
            if (g1 + h >= 0.0) {
                for (int64_t p = 0; p < np; ++p) P[p] = d[p];
                g1 = 0.0;
                for (int64_t p = 0; p < np; ++p) g1 += w[p] * b[p] * P[p];
            }
        }
        pair_wxw(W, n, pi, pj, np, P, V, wpw);
        double g2 = 0.0;
        for (int64_t p = 0; p < np; ++p) g2 += w[p] * P[p] * wpw[p];
        double kinkt;
        const double t = exact_step(c, P, w, np, lam, g1, g2, ks, &kinkt);
        for (int64_t p = 0; p < np; ++p) dprev[p] = d[p];
        if (t == 0.0) break;
        for (int64_t p = 0; p < np; ++p) {
            if (P[p] == 0.0) continue;
            const int64_t i = pi[p], j = pj[p];
            double nd;
            if (kinkt >= 0.0 && c[p] != 0.0 && -c[p] / P[p] == kinkt && sgn(c[p]) != sgn(P[p]))
                nd = -A[i * n + j]; /* lands on the kink: an exact zero */
            else
                nd = D[p] + t * P[p];
            if (zt[p] && c[p] != 0.0 && nd == D[p]) nd = -A[i * n + j]; /* zero snap */
            const double inc = nd - D[p];
            D[p] = nd;
            if (inc == 0.0) continue;
            for (int64_t k = 0; k < n; ++k) U[i * n + k] += inc * W[j * n + k];
            if (i != j)
                for (int64_t k = 0; k < n; ++k) U[j * n + k] += inc * W[i * n + k];
        }
    }
    free(d); free(dprev); free(P); free(b); free(c); free(w); free(wpw); free(zt); free(ks); free(V);
    return it;
}

/* ---------------------------------------------------------------------- */
/* a7. Armijo backtracking line search (Section 2 eq. Line-search; Section
 * 6.1.2 uses alpha_0 = 1, beta = 1/2 and positive definiteness).
 * READING: accept the first alpha = beta^t (t = 0..max_trials-1) for which
 * A + alpha Delta is positive definite and
 *     F(A + alpha Delta) <= F(A) + sigma alpha delta + eps_F,
 *     delta = tr(G Delta) + lambda (||A + Delta||_1 - ||A||_1),
 * with sigma = 1e-4 and the rounding allowance eps_F = 1e-12 max(|F(A)|, n):
 * near the optimum the predicted decrease falls below what an FP64 objective
 * can resolve, and without the allowance the test would reject unit steps on
 * rounding noise alone.  On success A is overwritten with A + alpha Delta and
 * F_inout with its objective.  Returns 0, or ORC_ELINESEARCH.              */
int orc_line_search(const double *S, const double *W, double *A, int64_t n, double lam,
                    const int32_t *pi, const int32_t *pj, int64_t np, const double *D,
                    double sigma, double beta, int max_trials, double *F_inout,
                    double *alpha_out, int *trials_out) {
    double delta = 0.0;
    for (int64_t p = 0; p < np; ++p) {
        int64_t i = pi[p], j = pj[p];
        double mult = (i == j) ? 1.0 : 2.0;
        double aij = A[i * n + j];
        delta += mult * ((S[i * n + j] - W[i * n + j]) * D[p] + lam * (fabs(aij + D[p]) - fabs(aij)));
    }
    double *T = (double *)malloc((size_t)(n * n) * sizeof(double));
    double epsF = 1e-12 * (fabs(*F_inout) > (double)n ? fabs(*F_inout) : (double)n);
    double alpha = 1.0;
    int ok = 0, t;
    for (t = 0; t < max_trials; ++t) {
        memcpy(T, A, (size_t)(n * n) * sizeof(double));
        for (int64_t p = 0; p < np; ++p) {
            int64_t i = pi[p], j = pj[p];
            T[i * n + j] = A[i * n + j] + alpha * D[p];
            T[j * n + i] = T[i * n + j];
        }
        double Ft;
        if (orc_objective(S, T, n, lam, &Ft) == 0 && Ft <= *F_inout + sigma * alpha * delta + epsF) {
            memcpy(A, T, (size_t)(n * n) * sizeof(double));
            *F_inout = Ft;
            ok = 1;
            break;
        }
        alpha *= beta;
    }
    free(T);
    if (alpha_out) *alpha_out = ok ? alpha : 0.0;
    if (trials_out) *trials_out = ok ? t + 1 : max_trials;
    return ok ? ORC_OK : ORC_ELINESEARCH;
}

/* ---------------------------------------------------------------------- */
/* a8. The ML-cycle, Algorithm 1 with nu = nu_c = 1 (Section 7), using the
 * dense one-block proximal Newton relaxation (QUIC-type, Sections 5.1-5.2).
 *
 * Relax(A, C_l):
 *   1. Cholesky of A, W = A^{-1}, G = S - W                   (eq. gradHes)
 *   2. free set F(A) restricted to C_l                         (eq. active_set)
 *   3. at l = 0: relative KKT of A; stop when <= tol (Section 3.2 last
 *      paragraph: the finest relaxation monitors convergence); keep this free
 *      set and |G| to define the next cycle's hierarchy (Section 7)
 *   4. Newton direction by nsweeps CD sweeps from Delta = 0   (eq. Quad_MLE_l1_prior)
 *   5. Armijo line search, A <- A + alpha Delta
 * Initial iterate A0 = diag(1 / (S_ii + lambda)) unless given; initial free set
 * {(i,j): |S_ij| > lambda} united with supp(A0) (Section 7 footnote) with
 * |G| = |S - A0^{-1}|.
 * READING: nsweeps = min(1 + floor(k/3), 10) for cycle k.
 *
 * one_level != 0: the one-level method the paper compares the multilevel
 * cycle against (Section 8: the same relaxation without the coarse levels):
 * every cycle is the single relaxation on the full free set (l = 0 only).
 * max_nnz: the largest nnz(A) (both triangles) seen at the start of a level-0
 * relaxation and at return (the paper's max-supp, sampled where the fine
 * free set is formed).
 *
 * continuation != 0: the continuation strategy (end of Section 2; the
 * schedule of Section 8): before the cycles at lambda, one level-0
 * relaxation at each of lambda_4 > lambda_3 > lambda_2 in that order, each
 * from the previous one's iterate (see orc_continuation_lambdas).  The free
 * set of the last one seeds the first cycle's hierarchy.  These relaxations
 * count in `relaxations` and in max_nnz, not in `cycles`; max_cycles bounds
 * the cycles at lambda only.
 *
 * inner = 0: the Newton direction by nsweeps CD sweeps (above); inner = 1: by
 * PCD-CG (orc_pcd) to the relative precision 1e-4 of Section 8, at most
 * 500 iterations.
 *
 * trace (optional, capacity trace_cap): after every relaxation, the objective
 * (at the lambda that relaxation used) and the level, as (F, level) pairs.    */
typedef struct {
    int status;
    int cycles;
    int relaxations;
    int ls_trials;
    double objective;
    double rel_kkt;
    double max_kkt;
    double logdet;
    int64_t nnz;
    int64_t ntrace;
    int64_t max_nnz;
} orc_info;

static int64_t count_nnz(const double *A, size_t nn) {
    int64_t c = 0;
    for (size_t t = 0; t < nn; ++t) c += A[t] != 0.0;
    return c;
}

/* The continuation's intermediate regularisation values (Section 8):
 * lambda_4 = (lambda_max + lambda) / 2 and lambda_3, lambda_2 linearly spaced
 * between lambda_4 and lambda_1 = lambda, i.e. lambda_s = lambda +
 * (s - 1)(lambda_4 - lambda) / 3.
 * READING: the paper takes lambda_4 = (1 + lambda) / 2 because its data are
 * normalised (diag S = 1), so every off-diagonal |S_ij| <= 1 and any lambda
 * >= 1 gives a diagonal minimiser.  For unnormalised S the same role is
 * played by lambda_max = max_{i != j} |S_ij|, the smallest lambda whose
 * minimiser is diagonal; lambda_max <= 1 on normalised data.  When
 * lambda_max <= lambda the solution at lambda is already diagonal and there
 * are no stages.
 * Writes lambda_4, lambda_3, lambda_2 to out[0..2]; returns the stage count
 * (3 or 0).                                                                  */
int orc_continuation_lambdas(const double *S, int64_t n, double lam, double *out) {
    double lmax = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            if (fabs(S[i * n + j]) > lmax) lmax = fabs(S[i * n + j]);
    if (!(lmax > lam)) return 0;
    const double l4 = 0.5 * (lmax + lam);
    for (int s = 4; s >= 2; --s) out[4 - s] = lam + (double)(s - 1) * (l4 - lam) / 3.0;
    return 3;
}

int orc_solve(const double *S, int64_t n, double lam, double tol, int max_cycles,
              const double *A0, double *A, double *W_out, orc_info *info,
              double *trace, int64_t trace_cap, int one_level, int continuation, int inner) {
    if (n < 1 || !(lam > 0.0)) return ORC_EINVAL;
    size_t nn = (size_t)(n * n);
    double *L = (double *)malloc(nn * sizeof(double));
    double *W = (double *)malloc(nn * sizeof(double));
    double *U = (double *)malloc(nn * sizeof(double));
    int64_t maxp = n * (n + 1) / 2;
    int32_t *fi = (int32_t *)malloc((size_t)maxp * sizeof(int32_t));
    int32_t *fj = (int32_t *)malloc((size_t)maxp * sizeof(int32_t));
    int32_t *ci = (int32_t *)malloc((size_t)maxp * sizeof(int32_t));
    int32_t *cj = (int32_t *)malloc((size_t)maxp * sizeof(int32_t));
    int32_t *pi = (int32_t *)malloc((size_t)maxp * sizeof(int32_t));
    int32_t *pj = (int32_t *)malloc((size_t)maxp * sizeof(int32_t));
    double *absg = (double *)malloc((size_t)maxp * sizeof(double));
    uint8_t *insupp = (uint8_t *)malloc((size_t)maxp);
    uint8_t *tag = (uint8_t *)malloc((size_t)maxp);
    double *D = (double *)malloc((size_t)maxp * sizeof(double));
    int status = ORC_EMAXITER;
    int relax = 0, lstrials = 0, cycles = 0;
    int64_t ntrace = 0, max_nnz = 0;
    double F = 0.0, relkkt = INFINITY, maxkkt = INFINITY, logdet = 0.0;

    if (A0) {
        memcpy(A, A0, nn * sizeof(double));
    } else {
        memset(A, 0, nn * sizeof(double));
        for (int64_t i = 0; i < n; ++i) {
            if (!(S[i * n + i] + lam > 0.0)) { status = ORC_ENOTPD; goto done; }
            A[i * n + i] = 1.0 / (S[i * n + i] + lam);
        }
    }
    /* initial free set and gradient */
    if (orc_cholesky(A, n, L) != 0) { status = ORC_ENOTPD; goto done; }
    orc_inverse_from_chol(L, n, W);
    int64_t nf = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i; j < n; ++j)
            if (fabs(S[i * n + j]) > lam || A[i * n + j] != 0.0) {
                fi[nf] = (int32_t)i;
                fj[nf] = (int32_t)j;
                absg[nf] = fabs(S[i * n + j] - W[i * n + j]);
                ++nf;
            }

    double stage_lam[3];
    const int nstage = continuation ? orc_continuation_lambdas(S, n, lam, stage_lam) : 0;
    /* k < 0: the continuation stages, one level-0 relaxation each at lambda_s */
    for (int k = -nstage; k < max_cycles; ++k) {
        const double lk = k < 0 ? stage_lam[k + nstage] : lam;
        if (k >= 0) cycles = k + 1;
        int nsweeps = k < 0 ? 1 : 1 + k / 3;
        if (nsweeps > 10) nsweeps = 10;
        for (int64_t p = 0; p < nf; ++p) insupp[p] = A[fi[p] * n + fj[p]] != 0.0;
        int L_levels = 1;
        orc_hierarchy(absg, insupp, nf, tag, &L_levels);
        if (one_level || k < 0) L_levels = 0;
        for (int l = L_levels; l >= 0; --l) {
            /* 1. factor, invert, objective */
            if (orc_cholesky(A, n, L) != 0) { status = ORC_ENOTPD; goto done; }
            logdet = orc_logdet_from_chol(L, n);
            orc_inverse_from_chol(L, n, W);
            double tr, l1;
            trace_and_l1(S, A, n, &tr, &l1);
            F = -logdet + tr + lk * l1;
            /* 2. free set restricted to C_l */
            int64_t np;
            if (l == 0) {
                const int64_t z = count_nnz(A, nn);
                if (z > max_nnz) max_nnz = z;
                np = orc_free_set(S, W, A, n, lk, NULL, NULL, 0, pi, pj);
                relkkt = orc_rel_kkt(S, W, A, n, lk, &maxkkt);
                /* 3. keep F_{k+1} and |G| for the next hierarchy */
                for (int64_t p = 0; p < np; ++p) {
                    fi[p] = pi[p];
                    fj[p] = pj[p];
                    absg[p] = fabs(S[pi[p] * n + pj[p]] - W[pi[p] * n + pj[p]]);
                }
                nf = np;
                if (k >= 0 && relkkt <= tol) { status = ORC_OK; goto done; }
            } else {
                int64_t nc = 0;
                for (int64_t p = 0; p < nf; ++p)
                    if (tag[p] >= l) { ci[nc] = fi[p]; cj[nc] = fj[p]; ++nc; }
                np = orc_free_set(S, W, A, n, lk, ci, cj, nc, pi, pj);
            }
            /* 4. Newton direction */
            memset(U, 0, nn * sizeof(double));
            memset(D, 0, (size_t)np * sizeof(double));
            if (inner == 1)
                orc_pcd(S, W, A, n, lk, pi, pj, np, 500, 1, 1e-4, D, U);
            else
                orc_cd_sweeps(S, W, A, n, lk, pi, pj, np, nsweeps, D, U);
            int moved = 0;
            for (int64_t p = 0; p < np; ++p) moved |= (D[p] != 0.0);
            /* 5. line search */
            if (moved) {
                double alpha;
                int tr_used;
                int rc = orc_line_search(S, W, A, n, lk, pi, pj, np, D, 1e-4, 0.5, 30, &F,
                                         &alpha, &tr_used);
                lstrials += tr_used;
                if (rc != ORC_OK) { status = rc; goto done; }
            }
            ++relax;
            if (trace && ntrace < trace_cap) {
                trace[2 * ntrace] = F;
                trace[2 * ntrace + 1] = (double)l;
                ++ntrace;
            }
        }
    }
done:
    if (status == ORC_OK || status == ORC_EMAXITER || status == ORC_ELINESEARCH) {
        if (orc_cholesky(A, n, L) == 0) {
            logdet = orc_logdet_from_chol(L, n);
            orc_inverse_from_chol(L, n, W);
            double tr, l1;
            trace_and_l1(S, A, n, &tr, &l1);
            F = -logdet + tr + lam * l1;
            relkkt = orc_rel_kkt(S, W, A, n, lam, &maxkkt);
            if (W_out) memcpy(W_out, W, nn * sizeof(double));
        }
    }
    if (info) {
        const int64_t nnz = count_nnz(A, nn);
        info->status = status;
        info->cycles = cycles;
        info->relaxations = relax;
        info->ls_trials = lstrials;
        info->objective = F;
        info->rel_kkt = relkkt;
        info->max_kkt = maxkkt;
        info->logdet = logdet;
        info->nnz = nnz;
        info->ntrace = ntrace;
        info->max_nnz = nnz > max_nnz ? nnz : max_nnz;
    }
    free(L); free(W); free(U); free(fi); free(fj); free(ci); free(cj); free(pi); free(pj);
    free(absg); free(insupp); free(tag); free(D);
    return status;
}

/* Screening: connected components of the graph with an edge (i, j), i != j,
 * wherever |S_ij| > lambda.  The minimiser is block diagonal over them and
 * each block is the minimiser of the problem on its sub-matrix of S (if A is
 * assembled from the blocks' minimisers, W = A^{-1} is block diagonal, and a
 * pair across blocks has A_ij = 0 and |G_ij| = |S_ij| <= lambda: the
 * zero-entry condition of eq. subgradient1; the minimiser is unique).
 * comp[i] = the smallest vertex of i's component, found by breadth-first
 * search from each unlabelled vertex in ascending order.  Returns the number
 * of components.                                                             */
int64_t orc_components(const double *S, int64_t n, double lam, int32_t *comp) {
    int32_t *queue = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int64_t ncomp = 0;
    for (int64_t i = 0; i < n; ++i) comp[i] = -1;
    for (int64_t r = 0; r < n; ++r) {
        if (comp[r] >= 0) continue;
        ++ncomp;
        int64_t head = 0, tail = 0;
        comp[r] = (int32_t)r;
        queue[tail++] = (int32_t)r;
        while (head < tail) {
            const int64_t v = queue[head++];
            for (int64_t u = 0; u < n; ++u) {
                if (u == v || comp[u] >= 0) continue;
                const double s = v < u ? S[v * n + u] : S[u * n + v];  /* upper triangle */
                if (fabs(s) > lam) {
                    comp[u] = (int32_t)r;
                    queue[tail++] = (int32_t)u;
                }
            }
        }
    }
    free(queue);
    return ncomp;
}

/* Relaxation count of trace entries written (for callers sizing buffers). */
int64_t orc_max_pairs(int64_t n) { return n * (n + 1) / 2; }

/* ---------------------------------------------------------------------- */
/* NEXT-4. BCD-IC (Section 6, Algorithm 2): the paper's relaxation for n
 * beyond dense memory, written here from its definitions on dense matrices.
 * The cheaper routes the paper takes at scale (only the columns I_j and N_j
 * of W, its appendix's formulas for the B_i from those columns) are not
 * taken: every quantity is formed from its definition.                     */

/* x = M^{-1} b for M = L L^T (L lower triangular, m x m). */
static void chol_solve(const double *L, int64_t m, const double *b, double *x) {
    for (int64_t i = 0; i < m; ++i) {
        double s = b[i];
        for (int64_t k = 0; k < i; ++k) s -= L[i * m + k] * x[k];
        x[i] = s / L[i * m + i];
    }
    for (int64_t i = m - 1; i >= 0; --i) {
        double s = x[i];
        for (int64_t k = i + 1; k < m; ++k) s -= L[k * m + i] * x[k];
        x[i] = s / L[i * m + i];
    }
}

/* Schur-complement log det (eq. Schurs_lemma, eq. logdet_blocks, eq.
 * Schurs_PDness).  The block "1" is the index set I (mask inI), "2" its
 * complement; Delta (pairs pi <= pj with values D, mirrored) must vanish on
 * the 22 block, as a block update's direction does:
 *   log det(A + alpha Delta) = log det A_22 + log det(B_0 + alpha B_1 + alpha^2 B_2),
 *   B_0 = A_11 - A_12 A_22^{-1} A_21,
 *   B_1 = Delta_11 - Delta_12 A_22^{-1} A_21 - A_12 A_22^{-1} Delta_21,
 *   B_2 = -Delta_12 A_22^{-1} Delta_21,
 * and A + alpha Delta is positive definite iff A_22 and the small matrix are.
 * A_22^{-1} A_21 and A_22^{-1} Delta_21 come from Cholesky solves with A_22.
 * Returns 0 with *ld set; 1 when A_22, 2 when the small matrix is not
 * positive definite; -1 when Delta is nonzero on the 22 block.             */
int orc_bcd_logdet(const double *A, int64_t n, const int32_t *pi, const int32_t *pj, int64_t np,
                   const double *D, const uint8_t *inI, double alpha, double *ld) {
    int64_t m1 = 0, m2 = 0;
    int64_t *i1 = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *i2 = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        if (inI[i]) i1[m1++] = i;
        else i2[m2++] = i;
    }
    double *Dl = (double *)calloc((size_t)(n * n), sizeof(double));
    const size_t s1 = (size_t)(m1 > 0 ? m1 : 1), s2 = (size_t)(m2 > 0 ? m2 : 1);
    double *A22 = (double *)malloc(s2 * s2 * sizeof(double));
    double *L22 = (double *)malloc(s2 * s2 * sizeof(double));
    double *Y = (double *)malloc(s2 * s1 * sizeof(double)); /* A_22^{-1} A_21, column c at Y[c m2] */
    double *Z = (double *)malloc(s2 * s1 * sizeof(double)); /* A_22^{-1} Delta_21 */
    double *rhs = (double *)malloc(s2 * sizeof(double));
    double *M = (double *)malloc(s1 * s1 * sizeof(double));
    double *LM = (double *)malloc(s1 * s1 * sizeof(double));
    int rc = 0;
    for (int64_t p = 0; p < np; ++p) {
        const int64_t i = pi[p], j = pj[p];
        if (!inI[i] && !inI[j] && D[p] != 0.0) { rc = -1; goto out; }
        Dl[i * n + j] = D[p];
        Dl[j * n + i] = D[p];
    }
    double ld22 = 0.0;
    if (m2 > 0) {
        for (int64_t a = 0; a < m2; ++a)
            for (int64_t c = 0; c < m2; ++c) A22[a * m2 + c] = A[i2[a] * n + i2[c]];
        if (orc_cholesky(A22, m2, L22) != 0) { rc = 1; goto out; }
        ld22 = orc_logdet_from_chol(L22, m2);
        for (int64_t c = 0; c < m1; ++c) {
            for (int64_t a = 0; a < m2; ++a) rhs[a] = A[i2[a] * n + i1[c]];
            chol_solve(L22, m2, rhs, Y + c * m2);
            for (int64_t a = 0; a < m2; ++a) rhs[a] = Dl[i2[a] * n + i1[c]];
            chol_solve(L22, m2, rhs, Z + c * m2);
        }
    }
    for (int64_t a = 0; a < m1; ++a)
        for (int64_t c = 0; c < m1; ++c) {
            const int64_t ia = i1[a], ic = i1[c];
            double b0 = A[ia * n + ic], b1 = Dl[ia * n + ic], b2 = 0.0;
            for (int64_t k = 0; k < m2; ++k) {
                const double a12 = A[ia * n + i2[k]], d12 = Dl[ia * n + i2[k]];
                b0 -= a12 * Y[c * m2 + k];
                b1 -= d12 * Y[c * m2 + k] + a12 * Z[c * m2 + k];
                b2 -= d12 * Z[c * m2 + k];
            }
            M[a * m1 + c] = b0 + alpha * b1 + alpha * alpha * b2;
        }
    if (m1 > 0 && orc_cholesky(M, m1, LM) != 0) { rc = 2; goto out; }
    *ld = ld22 + (m1 > 0 ? orc_logdet_from_chol(LM, m1) : 0.0);
out:
    free(i1); free(i2); free(Dl); free(A22); free(L22); free(Y); free(Z); free(rhs); free(M); free(LM);
    return rc;
}

/* One BCD-IC iteration (Algorithm 2) at lambda.  The columns are split into
 * the blocks I_j = [j b, min((j + 1) b, n)), treated in order (READING: the
 * paper clusters the columns with METIS, an external library, and allows any
 * partition; consecutive index ranges are the partition its Figure
 * fig:BCD_Sweep draws).  For each block, at the current iterate A:
 *   1. W = A^{-1} from the Cholesky factor (the algorithm solves linear
 *      systems for the columns I_j and N_j of W; all of W contains them);
 *   2. the block's free set (eq. active_set_j): the free pairs (eq.
 *      active_set, at the current A) with a row or a column in I_j, taken
 *      from the candidate list when one is given (Section 7: within C_l),
 *      else from all upper-triangle pairs;
 *   3. the Newton direction on those pairs from Delta = 0 (eq.
 *      sub_Quad_MLE_l1_prior): PCD-CG to the relative precision 1e-4 (the
 *      paper's block solver; inner = 1) or nsweeps CD sweeps (inner = 0);
 *   4. the line search along it, log det by eq. logdet_blocks, over the
 *      samples alpha_i = beta^i (beta = 1/2, at most 30):
 *      rule 1 (Section 6.1.2: the sample minimising F subject to positive
 *      definiteness): the first positive-definite alpha_i with F(alpha_i)
 *      <= F(A) + eps_F whose successor is not lower, F(alpha_{i+1}) >=
 *      F(alpha_i) (READING: F is convex along the ray, so the samples fall
 *      until the one before the first rise, the best of them);
 *      rule 0: the dense relaxation's Armijo test (orc_line_search), so that
 *      with one block holding every index the iteration is exactly the
 *      dense relaxation (Section 6.2: QUIC is BCD-IC with a single block).
 *      eps_F = 1e-12 max(|F(A)|, n) as there.
 * F_out: F of the final iterate.  Returns 0, ORC_ENOTPD (A not positive
 * definite) or ORC_ELINESEARCH; *moved = blocks with a nonzero direction;
 * *trials = objective evaluations of the line searches.                    */
int orc_bcd_iteration(const double *S, double *A, int64_t n, double lam, int64_t b,
                      const int32_t *cand_i, const int32_t *cand_j, int64_t ncand, int inner,
                      int nsweeps, int rule, double *F_out, int *trials, int *moved) {
    if (b < 1) b = n;
    const size_t nn = (size_t)(n * n);
    const int64_t maxp = cand_i ? (ncand > 0 ? ncand : 1) : n * (n + 1) / 2;
    double *L = (double *)malloc(nn * sizeof(double));
    double *W = (double *)malloc(nn * sizeof(double));
    double *U = (double *)malloc(nn * sizeof(double));
    double *T = (double *)malloc(nn * sizeof(double));
    int32_t *pi = (int32_t *)malloc((size_t)maxp * sizeof(int32_t));
    int32_t *pj = (int32_t *)malloc((size_t)maxp * sizeof(int32_t));
    double *D = (double *)malloc((size_t)maxp * sizeof(double));
    uint8_t *inI = (uint8_t *)malloc((size_t)n);
    int rc = ORC_OK, ntr = 0, nmv = 0;
    double F = 0.0;
    for (int64_t j0 = 0; j0 < n; j0 += b) {
        const int64_t j1 = j0 + b < n ? j0 + b : n;
        for (int64_t i = 0; i < n; ++i) inI[i] = i >= j0 && i < j1;
        if (orc_cholesky(A, n, L) != 0) { rc = ORC_ENOTPD; goto out; }
        orc_inverse_from_chol(L, n, W);
        double tr, l1;
        trace_and_l1(S, A, n, &tr, &l1);
        F = -orc_logdet_from_chol(L, n) + tr + lam * l1;
        int64_t np = 0;
        if (cand_i) {
            for (int64_t p = 0; p < ncand; ++p) {
                const int64_t i = cand_i[p], j = cand_j[p];
                if (!inI[i] && !inI[j]) continue;
                if (A[i * n + j] != 0.0 || fabs(S[i * n + j] - W[i * n + j]) > lam) {
                    pi[np] = (int32_t)i; pj[np] = (int32_t)j; ++np;
                }
            }
        } else {
            for (int64_t i = 0; i < n; ++i)
                for (int64_t j = i; j < n; ++j) {
                    if (!inI[i] && !inI[j]) continue;
                    if (A[i * n + j] != 0.0 || fabs(S[i * n + j] - W[i * n + j]) > lam) {
                        pi[np] = (int32_t)i; pj[np] = (int32_t)j; ++np;
                    }
                }
        }
        memset(U, 0, nn * sizeof(double));
        memset(D, 0, (size_t)(np > 0 ? np : 1) * sizeof(double));
        if (inner == 1)
            orc_pcd(S, W, A, n, lam, pi, pj, np, 500, 1, 1e-4, D, U);
        else
            orc_cd_sweeps(S, W, A, n, lam, pi, pj, np, nsweeps, D, U);
        int mv = 0;
        for (int64_t p = 0; p < np; ++p) mv |= D[p] != 0.0;
        if (!mv) continue;
        ++nmv;
        const double epsF = 1e-12 * (fabs(F) > (double)n ? fabs(F) : (double)n);
        double delta = 0.0;
        for (int64_t p = 0; p < np; ++p) {
            const int64_t i = pi[p], j = pj[p];
            const double mult = i == j ? 1.0 : 2.0, aij = A[i * n + j];
            delta += mult * ((S[i * n + j] - W[i * n + j]) * D[p] + lam * (fabs(aij + D[p]) - fabs(aij)));
        }
        /* F(A + alpha Delta) by eq. logdet_blocks; +inf when not positive definite */
        double alpha = 1.0, a_acc = 0.0, F_acc = 0.0, prevF = INFINITY, prevA = 0.0;
        int ok = 0;
        for (int t = 0; t < 30 && !ok; ++t, alpha *= 0.5) {
            memcpy(T, A, nn * sizeof(double));
            for (int64_t p = 0; p < np; ++p) {
                const int64_t i = pi[p], j = pj[p];
                T[i * n + j] = A[i * n + j] + alpha * D[p];
                T[j * n + i] = T[i * n + j];
            }
            double ldT = 0.0, Ft = INFINITY;
            ++ntr;
            if (orc_bcd_logdet(A, n, pi, pj, np, D, inI, alpha, &ldT) == 0) {
                double trT, l1T;
                trace_and_l1(S, T, n, &trT, &l1T);
                Ft = -ldT + trT + lam * l1T;
            }
            if (rule == 0) {
                if (Ft <= F + 1e-4 * alpha * delta + epsF) { ok = 1; a_acc = alpha; F_acc = Ft; }
            } else {
                if (prevF < INFINITY && prevF <= F + epsF && Ft >= prevF) { ok = 1; a_acc = prevA; F_acc = prevF; }
                prevF = Ft;
                prevA = alpha;
            }
        }
        if (!ok && rule != 0 && prevF <= F + epsF) {
            /* the samples fell to the last one: it is the best */
            ok = 1;
            a_acc = prevA;
            F_acc = prevF;
        }
        if (!ok) { rc = ORC_ELINESEARCH; goto out; }
        for (int64_t p = 0; p < np; ++p) {
            const int64_t i = pi[p], j = pj[p];
            A[i * n + j] = A[i * n + j] + a_acc * D[p];
            A[j * n + i] = A[i * n + j];
        }
        F = F_acc;
    }
    if (orc_cholesky(A, n, L) != 0) { rc = ORC_ENOTPD; goto out; }
    {
        double tr, l1;
        trace_and_l1(S, A, n, &tr, &l1);
        F = -orc_logdet_from_chol(L, n) + tr + lam * l1;
    }
out:
    if (F_out) *F_out = F;
    if (trials) *trials = ntr;
    if (moved) *moved = nmv;
    free(L); free(W); free(U); free(T); free(pi); free(pj); free(D); free(inI);
    return rc;
}

/* ML-BCD: the ML-cycle of orc_solve (Algorithm 1 with nu = nu_c = 1, the
 * hierarchy of Section 7, the Section 8 KKT stop) with one BCD-IC iteration
 * (orc_bcd_iteration, blocks of b columns) as the relaxation on C_l, the
 * combination the paper measures (Section 7: BCD-IC as the relaxation, the
 * block free sets within C_l).  At level 0 the block free sets come from all
 * pairs; at level l > 0 from the candidates of C_l (the previous fine free
 * set's pairs with tag >= l).  inner, rule: as in orc_bcd_iteration; CD
 * sweeps take nsweeps = min(1 + floor(k/3), 10) in cycle k as orc_solve does.
 * one_level != 0: the level-0 relaxation only (BCD-IC alone).              */
int orc_solve_bcd(const double *S, int64_t n, double lam, double tol, int max_cycles,
                  const double *A0, double *A, orc_info *info, int64_t b, int inner, int rule,
                  int one_level) {
    if (n < 1 || !(lam > 0.0)) return ORC_EINVAL;
    const size_t nn = (size_t)(n * n);
    const int64_t maxp = n * (n + 1) / 2;
    double *L = (double *)malloc(nn * sizeof(double));
    double *W = (double *)malloc(nn * sizeof(double));
    int32_t *fi = (int32_t *)malloc((size_t)maxp * sizeof(int32_t));
    int32_t *fj = (int32_t *)malloc((size_t)maxp * sizeof(int32_t));
    int32_t *ci = (int32_t *)malloc((size_t)maxp * sizeof(int32_t));
    int32_t *cj = (int32_t *)malloc((size_t)maxp * sizeof(int32_t));
    double *absg = (double *)malloc((size_t)maxp * sizeof(double));
    uint8_t *insupp = (uint8_t *)malloc((size_t)maxp);
    uint8_t *tag = (uint8_t *)malloc((size_t)maxp);
    int status = ORC_EMAXITER, relax = 0, lstrials = 0, cycles = 0;
    int64_t max_nnz = 0, nf = 0;
    double F = 0.0, relkkt = INFINITY, maxkkt = INFINITY, logdet = 0.0;
    if (A0) {
        memcpy(A, A0, nn * sizeof(double));
    } else {
        memset(A, 0, nn * sizeof(double));
        for (int64_t i = 0; i < n; ++i) {
            if (!(S[i * n + i] + lam > 0.0)) { status = ORC_ENOTPD; goto done; }
            A[i * n + i] = 1.0 / (S[i * n + i] + lam);
        }
    }
    if (orc_cholesky(A, n, L) != 0) { status = ORC_ENOTPD; goto done; }
    orc_inverse_from_chol(L, n, W);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i; j < n; ++j)
            if (fabs(S[i * n + j]) > lam || A[i * n + j] != 0.0) {
                fi[nf] = (int32_t)i; fj[nf] = (int32_t)j;
                absg[nf] = fabs(S[i * n + j] - W[i * n + j]);
                ++nf;
            }
    for (int k = 0; k < max_cycles; ++k) {
        cycles = k + 1;
        int nsweeps = 1 + k / 3;
        if (nsweeps > 10) nsweeps = 10;
        for (int64_t p = 0; p < nf; ++p) insupp[p] = A[fi[p] * n + fj[p]] != 0.0;
        int L_levels = 1;
        orc_hierarchy(absg, insupp, nf, tag, &L_levels);
        if (one_level) L_levels = 0;
        for (int l = L_levels; l >= 0; --l) {
            const int32_t *qi = NULL, *qj = NULL;
            int64_t nq = 0;
            if (l == 0) {
                if (orc_cholesky(A, n, L) != 0) { status = ORC_ENOTPD; goto done; }
                orc_inverse_from_chol(L, n, W);
                const int64_t z = count_nnz(A, nn);
                if (z > max_nnz) max_nnz = z;
                nf = orc_free_set(S, W, A, n, lam, NULL, NULL, 0, fi, fj);
                for (int64_t p = 0; p < nf; ++p) absg[p] = fabs(S[fi[p] * n + fj[p]] - W[fi[p] * n + fj[p]]);
                relkkt = orc_rel_kkt(S, W, A, n, lam, &maxkkt);
                if (relkkt <= tol) { status = ORC_OK; goto done; }
            } else {
                for (int64_t p = 0; p < nf; ++p)
                    if (tag[p] >= l) { ci[nq] = fi[p]; cj[nq] = fj[p]; ++nq; }
                qi = ci;
                qj = cj;
            }
            int tr = 0, mv = 0;
            const int rc = orc_bcd_iteration(S, A, n, lam, b, qi, qj, nq, inner, nsweeps, rule, &F, &tr, &mv);
            lstrials += tr;
            if (rc != ORC_OK) { status = rc; goto done; }
            ++relax;
        }
    }
done:
    if (status == ORC_OK || status == ORC_EMAXITER || status == ORC_ELINESEARCH) {
        if (orc_cholesky(A, n, L) == 0) {
            logdet = orc_logdet_from_chol(L, n);
            orc_inverse_from_chol(L, n, W);
            double tr, l1;
            trace_and_l1(S, A, n, &tr, &l1);
            F = -logdet + tr + lam * l1;
            relkkt = orc_rel_kkt(S, W, A, n, lam, &maxkkt);
        }
    }
    if (info) {
        const int64_t nnz = count_nnz(A, nn);
        info->status = status;
        info->cycles = cycles;
        info->relaxations = relax;
        info->ls_trials = lstrials;
        info->objective = F;
        info->rel_kkt = relkkt;
        info->max_kkt = maxkkt;
        info->logdet = logdet;
        info->nnz = nnz;
        info->ntrace = 0;
        info->max_nnz = nnz > max_nnz ? nnz : max_nnz;
    }
    free(L); free(W); free(fi); free(fj); free(ci); free(cj); free(absg); free(insupp); free(tag);
    return status;
}

/* The diagonal block W_11 = (A^{-1})_{I I} of a block from the columns of W
 * in the block's C-neighbourhood only (appendix sec:reducingGradient, eq.
 * reducingGradients1-2): block row I of A W = I reads A_11 W_11 + K = I with
 * K = A_12 W_21, and A_12 is nonzero only in the neighbourhood's columns when
 * supp(A) lies in C, so
 *     K_ac = sum_{k in N} A_{a k} W_{k c}   (W_{k c} = W_{c k}: column k of W),
 *     W_11 = A_11^{-1} (I - K)              (Cholesky solves with A_11).
 * READING: the neighbourhood N = {k not in I : (i, k) in C for some i in I}
 * (the printed eq. extended_set_C quantifies over the wrong index: read
 * literally it holds every index outside I through the diagonal pairs).
 * inN: the mask of N; WN: an n x n array whose columns k in N hold column k
 * of A^{-1} (other columns are not read).  W11: m1 x m1 in the order of I.
 * Returns 0; 1 when A_11 is not positive definite; -1 when A_12 has a
 * nonzero outside N (the support is not within C).                         */
int orc_bcd_w11(const double *A, int64_t n, const uint8_t *inI, const uint8_t *inN, const double *WN,
                double *W11) {
    int64_t m1 = 0;
    int64_t *i1 = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i)
        if (inI[i]) i1[m1++] = i;
    const size_t s1 = (size_t)(m1 > 0 ? m1 : 1);
    double *A11 = (double *)malloc(s1 * s1 * sizeof(double));
    double *L11 = (double *)malloc(s1 * s1 * sizeof(double));
    double *rhs = (double *)malloc(s1 * sizeof(double));
    double *x = (double *)malloc(s1 * sizeof(double));
    int rc = 0;
    for (int64_t a = 0; a < m1; ++a)
        for (int64_t k = 0; k < n; ++k)
            if (!inI[k] && !inN[k] && A[i1[a] * n + k] != 0.0) { rc = -1; goto out; }
    for (int64_t a = 0; a < m1; ++a)
        for (int64_t c = 0; c < m1; ++c) A11[a * m1 + c] = A[i1[a] * n + i1[c]];
    if (m1 > 0 && orc_cholesky(A11, m1, L11) != 0) { rc = 1; goto out; }
    for (int64_t c = 0; c < m1; ++c) {
        /* column c of I - K */
        for (int64_t a = 0; a < m1; ++a) {
            double kac = 0.0;
            for (int64_t k = 0; k < n; ++k)
                if (inN[k]) kac += A[i1[a] * n + k] * WN[i1[c] * n + k];
            rhs[a] = (a == c ? 1.0 : 0.0) - kac;
        }
        chol_solve(L11, m1, rhs, x);
        for (int64_t a = 0; a < m1; ++a) W11[a * m1 + c] = x[a];
    }
out:
    free(i1); free(A11); free(L11); free(rhs); free(x);
    return rc;
}
