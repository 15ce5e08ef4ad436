/*
 * FP64 CPU oracle for fast binary semi-supervised discriminant analysis
 * (FSDA, Algorithm 7 of Tavernier et al., "Fast semi-supervised discriminant
 * analysis for binary classification of large data-sets").
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file; the product (the CUDA library) never does
 * and shares no code with it.
 *
 * It follows the paper's statement of the method, in its order and notation:
 *
 *   mean labelled sample      l mu_l = X^T 1_l                      Alg. 7 step 3
 *   Laplacian                 L = D - S,  D_ii = sum_j s_ij          Sec. 2.3
 *   operator (paper form)     B p = (X - 1 mu_l^T)^T M X p,
 *                             M = (1 - alpha) P_l + alpha L          Alg. 7 step 4, eq. (7)
 *     evaluated as            u = X p,  v = omega P_l u + alpha L u,
 *                             B p = X^T v - mu_l <1, v>              Sec. 3.2.3 (second identity)
 *   right-hand side           b = (X - 1 mu_l^T)^T [W 0; 0 0] X r    Alg. 7 step 4
 *   conjugate gradient        Algorithm 2
 *   shifted CG                Algorithm 3, with the readings:
 *     - base system B + sigma0 I, sigma0 = min beta; the recurrences use the
 *       relative shifts beta - sigma0 (the base B alone is singular);
 *     - the shift-coefficient update uses the new CG coefficient:
 *       alpha^b_{i+1} = alpha_{i+1} (zeta^b_{i+1} / zeta^b_i)^2
 *       (the printed alpha_i is an index slip; with it the shifted iterates
 *       stop matching per-shift CG);
 *     - "||r|| < tol" is read relative: |zeta^b| ||r|| < tol ||b||; the loop
 *       runs until every shift has stopped or max_iter is reached.
 *   omega is the weight of the labelled total scatter; the paper's value is
 *   1 - alpha and the caller passes it explicitly.
 *
 * Parallel loops (OpenMP) only split independent output elements; every
 * sum runs in a fixed order, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n, d;
    const int64_t *xp; const int32_t *xc; const double *xv;   /* X, CSR, n x d */
    const int64_t *sp; const int32_t *sc; const double *sv;   /* S, CSR, n x n */
    const int8_t *y;                                          /* +1 / -1 / 0   */
    double alpha, omega;
    /* owned */
    int64_t *tp; int32_t *tr; double *tv;                      /* X^T as CSR (d x n) */
    double *deg;                                               /* D_ii = sum_j s_ij  */
    double *mu;                                                /* mu_l               */
    double *u, *v;                                             /* work, n each       */
    double ell, npos, nneg;
} oracle_problem;

int oracle_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
    return omp_get_max_threads();
#else
    (void)t;
    return 1;
#endif
}

static double dot(int64_t m, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += a[i] * b[i];
    return s;
}

/* u = X p */
static void x_mul(const oracle_problem *P, const double *p, double *u)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < P->n; ++i) {
        double s = 0.0;
        for (int64_t e = P->xp[i]; e < P->xp[i + 1]; ++e) s += P->xv[e] * p[P->xc[e]];
        u[i] = s;
    }
}

/* q = X^T v */
static void xt_mul(const oracle_problem *P, const double *v, double *q)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < P->d; ++j) {
        double s = 0.0;
        for (int64_t e = P->tp[j]; e < P->tp[j + 1]; ++e) s += P->tv[e] * v[P->tr[e]];
        q[j] = s;
    }
}

void oracle_destroy(oracle_problem *P)
{
    if (!P) return;
    free(P->tp); free(P->tr); free(P->tv); free(P->deg); free(P->mu); free(P->u); free(P->v);
    free(P);
}

/* Builds the problem; the caller keeps the input arrays alive.  NULL on error. */
oracle_problem *oracle_create(int64_t n, int64_t d,
                              const int64_t *xp, const int32_t *xc, const double *xv,
                              const int64_t *sp, const int32_t *sc, const double *sv,
                              const int8_t *y, double alpha, double omega)
{
    oracle_problem *P = (oracle_problem *)calloc(1, sizeof(oracle_problem));
    if (!P) return NULL;
    P->n = n; P->d = d; P->xp = xp; P->xc = xc; P->xv = xv; P->sp = sp; P->sc = sc; P->sv = sv;
    P->y = y; P->alpha = alpha; P->omega = omega;
    int64_t nnz = xp[n];
    P->tp = (int64_t *)calloc((size_t)d + 1, sizeof(int64_t));
    P->tr = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    P->tv = (double *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
    P->deg = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    P->mu = (double *)calloc((size_t)(d > 0 ? d : 1), sizeof(double));
    P->u = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    P->v = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!P->tp || !P->tr || !P->tv || !P->deg || !P->mu || !P->u || !P->v) {
        oracle_destroy(P);
        return NULL;
    }
    /* transpose by counting sort: rows stay ascending inside each column */
    for (int64_t e = 0; e < nnz; ++e) {
        if (xc[e] < 0 || xc[e] >= d) { oracle_destroy(P); return NULL; }
        P->tp[xc[e] + 1]++;
    }
    for (int64_t j = 0; j < d; ++j) P->tp[j + 1] += P->tp[j];
    int64_t *fill = (int64_t *)malloc(((size_t)d + 1) * sizeof(int64_t));
    if (!fill) { oracle_destroy(P); return NULL; }
    memcpy(fill, P->tp, ((size_t)d + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = xp[i]; e < xp[i + 1]; ++e) {
            int64_t k = fill[xc[e]]++;
            P->tr[k] = (int32_t)i;
            P->tv[k] = xv[e];
        }
    free(fill);
    /* degrees of the similarity graph */
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t e = sp[i]; e < sp[i + 1]; ++e) s += sv[e];
        P->deg[i] = s;
    }
    /* l mu_l = X^T 1_l (Alg. 7 step 3) */
    double ell = 0.0, np_ = 0.0, nn_ = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        P->u[i] = y[i] != 0 ? 1.0 : 0.0;
        ell += P->u[i];
        np_ += y[i] > 0 ? 1.0 : 0.0;
        nn_ += y[i] < 0 ? 1.0 : 0.0;
    }
    P->ell = ell; P->npos = np_; P->nneg = nn_;
    xt_mul(P, P->u, P->mu);
    if (ell > 0)
        for (int64_t j = 0; j < d; ++j) P->mu[j] /= ell;
    return P;
}

/* The operator of CSR-SDA's regression step (Algorithm 5, line 5: shifted CG
 * on (X^T X + beta I) w = X^T z): B = X^T X, i.e. the operator above with no
 * graph, every row labelled (P_l = I), alpha = 0, omega = 1 and no centring
 * (mu_l = 0).  sp_zero: n + 1 zero row pointers, y_ones: n labels +1, kept
 * alive by the caller.  NULL on error. */
oracle_problem *oracle_create_regression(int64_t n, int64_t d, const int64_t *xp, const int32_t *xc,
                                         const double *xv, const int64_t *sp_zero, const int8_t *y_ones)
{
    oracle_problem *P = oracle_create(n, d, xp, xc, xv, sp_zero, NULL, NULL, y_ones, 0.0, 1.0);
    if (P) memset(P->mu, 0, (size_t)(d > 0 ? d : 1) * sizeof(double));
    return P;
}

/* Class counts and means: mu_l, mu_+ = X^T 1_+ / N_+, mu_- = X^T 1_- / N_-. */
void oracle_class_means(const oracle_problem *P, double *mu_l, double *mu_pos, double *mu_neg,
                        double *counts /* [ell, N+, N-] */)
{
    double *ind = (double *)malloc((size_t)(P->n > 0 ? P->n : 1) * sizeof(double));
    memcpy(mu_l, P->mu, (size_t)P->d * sizeof(double));
    for (int64_t i = 0; i < P->n; ++i) ind[i] = P->y[i] > 0 ? 1.0 : 0.0;
    xt_mul(P, ind, mu_pos);
    for (int64_t i = 0; i < P->n; ++i) ind[i] = P->y[i] < 0 ? 1.0 : 0.0;
    xt_mul(P, ind, mu_neg);
    for (int64_t j = 0; j < P->d; ++j) {
        mu_pos[j] = P->npos > 0 ? mu_pos[j] / P->npos : 0.0;
        mu_neg[j] = P->nneg > 0 ? mu_neg[j] / P->nneg : 0.0;
    }
    counts[0] = P->ell; counts[1] = P->npos; counts[2] = P->nneg;
    free(ind);
}

/* q = (B + sigma I) p with B in the paper's form (X - 1 mu_l^T)^T M X. */
void oracle_apply(oracle_problem *P, double sigma, const double *p, double *q)
{
    double *u = P->u, *v = P->v;
    x_mul(P, p, u);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < P->n; ++i) {
        double su = 0.0;
        for (int64_t e = P->sp[i]; e < P->sp[i + 1]; ++e) su += P->sv[e] * u[P->sc[e]];
        double lu = P->deg[i] * u[i] - su;                     /* (L u)_i */
        double pu = P->y[i] != 0 ? u[i] : 0.0;                  /* (P_l u)_i */
        v[i] = P->omega * pu + P->alpha * lu;
    }
    double sum_v = 0.0;
    for (int64_t i = 0; i < P->n; ++i) sum_v += v[i];
    xt_mul(P, v, q);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < P->d; ++j) q[j] = q[j] - P->mu[j] * sum_v + sigma * p[j];
}

/* b = (X - 1 mu_l^T)^T [W 0; 0 0] X r with W block-diagonal, 1/N_c in class c (Alg. 7 step 4). */
void oracle_rhs_from_r(oracle_problem *P, const double *r, double *b)
{
    double *u = P->u, *z = P->v;
    x_mul(P, r, u);
    double sp_ = 0.0, sn_ = 0.0;
    for (int64_t i = 0; i < P->n; ++i) {
        if (P->y[i] > 0) sp_ += u[i];
        else if (P->y[i] < 0) sn_ += u[i];
    }
    double mp = P->npos > 0 ? sp_ / P->npos : 0.0, mn = P->nneg > 0 ? sn_ / P->nneg : 0.0;
    for (int64_t i = 0; i < P->n; ++i) z[i] = P->y[i] > 0 ? mp : (P->y[i] < 0 ? mn : 0.0);
    double sum_z = 0.0;
    for (int64_t i = 0; i < P->n; ++i) sum_z += z[i];
    xt_mul(P, z, b);
    for (int64_t j = 0; j < P->d; ++j) b[j] -= P->mu[j] * sum_z;
}

/* s = X w (Sec. 4: the rating of the samples). */
void oracle_project(const oracle_problem *P, const double *w, double *s) { x_mul(P, w, s); }

/*
 * Algorithm 2 on (B + beta I) w = b.  fixed_iters > 0 runs exactly that many
 * iterations and ignores tol.  Returns 0, or -1 on breakdown (<p,q> <= 0 or
 * not finite), -2 on allocation failure.
 */
int oracle_cg(oracle_problem *P, const double *b, double beta, double tol, int max_iter,
              int fixed_iters, double *w, int *iters, double *res_est)
{
    int64_t d = P->d;
    double *r = (double *)malloc((size_t)d * sizeof(double));
    double *p = (double *)malloc((size_t)d * sizeof(double));
    double *q = (double *)malloc((size_t)d * sizeof(double));
    if (!r || !p || !q) { free(r); free(p); free(q); return -2; }
    memcpy(r, b, (size_t)d * sizeof(double));
    memcpy(p, b, (size_t)d * sizeof(double));
    memset(w, 0, (size_t)d * sizeof(double));
    double rr = dot(d, r, r), bnorm = sqrt(rr);
    int limit = fixed_iters > 0 ? fixed_iters : max_iter, i = 0, rc = 0;
    if (fixed_iters <= 0 && bnorm == 0.0) limit = 0;
    for (i = 0; i < limit; ++i) {
        oracle_apply(P, beta, p, q);
        double pq = dot(d, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { rc = -1; break; }
        double gamma = -rr / pq;
        for (int64_t j = 0; j < d; ++j) w[j] -= gamma * p[j];
        for (int64_t j = 0; j < d; ++j) r[j] += gamma * q[j];
        double rr_new = dot(d, r, r);
        if (fixed_iters <= 0 && sqrt(rr_new) < tol * bnorm) { rr = rr_new; ++i; break; }
        /* a vanished residual: w is exact, nothing is left to iterate on */
        if (rr_new == 0.0) { rr = rr_new; ++i; break; }
        double a = rr_new / rr;
        for (int64_t j = 0; j < d; ++j) p[j] = r[j] + a * p[j];
        rr = rr_new;
    }
    *iters = i;
    *res_est = bnorm > 0 ? sqrt(rr) / bnorm : 0.0;
    free(r); free(p); free(q);
    return rc;
}

/*
 * Algorithm 3: (B + beta_s I) W_s = b for every shift, W is [n_shifts][d].
 * iters[s] is the iteration at which shift s stopped; res_est[s] its
 * estimated relative residual |zeta_s| ||r|| / ||b||.  *total is the number
 * of operator applications.  Returns 0, -1 on breakdown, -2 on allocation
 * failure, -3 if a shift is below the smallest one (impossible by
 * construction).
 */
int oracle_shifted_cg(oracle_problem *P, const double *b, const double *betas, int ns,
                      double tol, int max_iter, int fixed_iters,
                      double *W, int *iters, double *res_est, int *total)
{
    int64_t d = P->d;
    double sigma0 = betas[0];
    for (int s = 1; s < ns; ++s) sigma0 = betas[s] < sigma0 ? betas[s] : sigma0;
    double *r = (double *)malloc((size_t)d * sizeof(double));
    double *p = (double *)malloc((size_t)d * sizeof(double));
    double *q = (double *)malloc((size_t)d * sizeof(double));
    double *Ps = (double *)malloc((size_t)d * ns * sizeof(double));
    double *zp = (double *)malloc((size_t)ns * sizeof(double));   /* zeta_{i-1} */
    double *z = (double *)malloc((size_t)ns * sizeof(double));    /* zeta_i     */
    double *zn = (double *)malloc((size_t)ns * sizeof(double));   /* zeta_{i+1} */
    double *gs = (double *)malloc((size_t)ns * sizeof(double));   /* gamma^b_i  */
    double *as = (double *)malloc((size_t)ns * sizeof(double));   /* alpha^b    */
    int *act = (int *)malloc((size_t)ns * sizeof(int));
    if (!r || !p || !q || !Ps || !zp || !z || !zn || !gs || !as || !act) {
        free(r); free(p); free(q); free(Ps); free(zp); free(z); free(zn); free(gs); free(as); free(act);
        return -2;
    }
    memcpy(r, b, (size_t)d * sizeof(double));
    memcpy(p, b, (size_t)d * sizeof(double));
    memset(W, 0, (size_t)d * ns * sizeof(double));
    for (int s = 0; s < ns; ++s) {
        memcpy(Ps + (int64_t)s * d, b, (size_t)d * sizeof(double));
        zp[s] = 1.0; z[s] = 1.0; as[s] = 0.0; act[s] = 1; iters[s] = 0;
    }
    double rr = dot(d, r, r), bnorm = sqrt(rr);
    double alpha = 0.0, gamma_prev = 1.0;
    int limit = fixed_iters > 0 ? fixed_iters : max_iter, rc = 0, i, nact = ns;
    if (fixed_iters <= 0 && bnorm == 0.0) nact = 0;
    for (i = 0; i < limit && nact > 0; ++i) {
        oracle_apply(P, sigma0, p, q);
        double pq = dot(d, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { rc = -1; break; }
        double gamma = -rr / pq;
        for (int s = 0; s < ns; ++s) {
            if (!act[s]) continue;
            double delta = betas[s] - sigma0;
            double den = gamma * alpha * (zp[s] - z[s]) + zp[s] * gamma_prev * (1.0 - delta * gamma);
            zn[s] = zp[s] * z[s] * gamma_prev / den;
            gs[s] = gamma * zn[s] / z[s];
        }
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < d; ++j)
            for (int s = 0; s < ns; ++s)
                if (act[s]) W[(int64_t)s * d + j] -= gs[s] * Ps[(int64_t)s * d + j];
        for (int64_t j = 0; j < d; ++j) r[j] += gamma * q[j];
        double rr_new = dot(d, r, r);
        double alpha_new = rr_new / rr;
        for (int64_t j = 0; j < d; ++j) p[j] = r[j] + alpha_new * p[j];
        for (int s = 0; s < ns; ++s) {
            if (!act[s]) continue;
            double ratio = zn[s] / z[s];
            as[s] = alpha_new * ratio * ratio;
        }
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < d; ++j)
            for (int s = 0; s < ns; ++s)
                if (act[s]) Ps[(int64_t)s * d + j] = zn[s] * r[j] + as[s] * Ps[(int64_t)s * d + j];
        double rnorm = sqrt(rr_new);
        for (int s = 0; s < ns; ++s) {
            if (!act[s]) continue;
            zp[s] = z[s];
            z[s] = zn[s];
            iters[s] = i + 1;
            res_est[s] = bnorm > 0 ? fabs(z[s]) * rnorm / bnorm : 0.0;
            if (fixed_iters <= 0 && (fabs(z[s]) * rnorm < tol * bnorm || !(fabs(z[s]) > 0.0))) {
                act[s] = 0;
                --nact;
            }
        }
        gamma_prev = gamma;
        alpha = alpha_new;
        rr = rr_new;
        /* a vanished residual: every shift's W_s is exact (its residual is
           zeta_s r = 0), nothing is left to iterate on */
        if (rr_new == 0.0) { ++i; break; }
    }
    if (bnorm == 0.0)
        for (int s = 0; s < ns; ++s) res_est[s] = 0.0;
    *total = i;
    free(r); free(p); free(q); free(Ps); free(zp); free(z); free(zn); free(gs); free(as); free(act);
    return rc;
}
