/*
 * Native helpers of the seeded input generator (synth.py).  They build the
 * *inputs* of the solver and hold none of its arithmetic:
 *
 *  - synth_knn_jaccard: k-nearest-neighbour lists of the rows of a sparse
 *    sample x feature matrix under the Jaccard (Tanimoto) similarity of their
 *    binary supports (the similarity graph S of Sec. 2.3-2.4; Tanimoto kNN in
 *    Sec. 5.1).
 *  - synth_row_counts / synth_fill_rows: the rows of X for the large
 *    workloads (Poisson nonzero counts, Zipf-popular columns, binary or
 *    geometric count values), one counter-based random stream per row.
 *  - synth_planted: binary targets from a planted sparse linear model, one
 *    random stream per target.
 *
 * Every random draw comes from splitmix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014) on a per-row or
 * per-target counter, so the output never depends on the thread count.
 *
 * kNN: candidates of row i are the rows j != i that share at least one
 * feature whose column count is <= cap.  With cap >= n every shared feature
 * counts, and the lists are the exact kNN among rows with nonzero
 * similarity.  Neighbours are ranked by (similarity descending, row index
 * ascending); similarity 0 never makes a neighbour.
 */
#include <stdint.h>
#include <stdlib.h>
#include <math.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int64_t inter_sorted(const int32_t *a, int64_t na, const int32_t *b, int64_t nb)
{
    int64_t i = 0, j = 0, c = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) {
            ++i;
        } else if (a[i] > b[j]) {
            ++j;
        } else {
            ++c; ++i; ++j;
        }
    }
    return c;
}

/* Returns 0 on success, -1 on allocation failure, -2 on bad arguments. */
int synth_knn_jaccard(int64_t n, int64_t d, const int64_t *rp, const int32_t *ci,
                      int32_t k, int64_t cap, int32_t *nbr, double *sim, int32_t nthreads)
{
    if (n < 0 || d < 0 || k <= 0) return -2;
    int64_t nnz = rp[n];
    int64_t *cnt = (int64_t *)calloc((size_t)d + 1, sizeof(int64_t));
    if (!cnt) return -1;
    for (int64_t e = 0; e < nnz; ++e) {
        if (ci[e] < 0 || ci[e] >= d) { free(cnt); return -2; }
        cnt[ci[e]]++;
    }
    /* inverted lists of the candidate columns only */
    int64_t *iptr = (int64_t *)malloc(((size_t)d + 1) * sizeof(int64_t));
    if (!iptr) { free(cnt); return -1; }
    iptr[0] = 0;
    for (int64_t f = 0; f < d; ++f) iptr[f + 1] = iptr[f] + (cnt[f] <= cap ? cnt[f] : 0);
    int32_t *irow = (int32_t *)malloc((size_t)(iptr[d] > 0 ? iptr[d] : 1) * sizeof(int32_t));
    int64_t *fill = (int64_t *)malloc(((size_t)d + 1) * sizeof(int64_t));
    if (!irow || !fill) { free(cnt); free(iptr); free(irow); free(fill); return -1; }
    memcpy(fill, iptr, (size_t)d * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            if (cnt[ci[e]] <= cap) irow[fill[ci[e]]++] = (int32_t)i;
    free(fill);

    int failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        int32_t *mark = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        int32_t *cand = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        int32_t *bj = (int32_t *)malloc((size_t)k * sizeof(int32_t));
        double *bs = (double *)malloc((size_t)k * sizeof(double));
        if (!mark || !cand || !bj || !bs) {
#pragma omp atomic write
            failed = 1;
        } else {
            for (int64_t i = 0; i < n; ++i) mark[i] = -1;
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = 0; i < n; ++i) {
                int64_t nc = 0;
                for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
                    int32_t f = ci[e];
                    if (cnt[f] > cap) continue;
                    for (int64_t t = iptr[f]; t < iptr[f + 1]; ++t) {
                        int32_t j = irow[t];
                        if (j == i || mark[j] == (int32_t)i) continue;
                        mark[j] = (int32_t)i;
                        cand[nc++] = j;
                    }
                }
                int32_t nb = 0;
                int64_t li = rp[i + 1] - rp[i];
                for (int64_t c = 0; c < nc; ++c) {
                    int32_t j = cand[c];
                    int64_t lj = rp[j + 1] - rp[j];
                    int64_t in = inter_sorted(ci + rp[i], li, ci + rp[j], lj);
                    if (in == 0) continue;
                    double s = (double)in / (double)(li + lj - in);
                    /* insert into the sorted top-k list: (s desc, j asc) */
                    int32_t pos = nb;
                    while (pos > 0 && (bs[pos - 1] < s || (bs[pos - 1] == s && bj[pos - 1] > j))) --pos;
                    if (pos >= k) continue;
                    int32_t last = nb < k ? nb : k - 1;
                    for (int32_t m = last; m > pos; --m) { bs[m] = bs[m - 1]; bj[m] = bj[m - 1]; }
                    bs[pos] = s; bj[pos] = j;
                    if (nb < k) ++nb;
                }
                for (int32_t m = 0; m < k; ++m) {
                    nbr[i * (int64_t)k + m] = m < nb ? bj[m] : -1;
                    sim[i * (int64_t)k + m] = m < nb ? bs[m] : 0.0;
                }
            }
        }
        free(mark); free(cand); free(bj); free(bs);
    }
    free(cnt); free(iptr); free(irow);
    return failed ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* counter-based random stream                                               */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t s; } rng_t;

static uint64_t rng_next(rng_t *r)
{
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* stream `idx` of generator `seed` */
static rng_t rng_stream(uint64_t seed, uint64_t idx, uint64_t tag)
{
    rng_t r;
    r.s = seed * 0xD1B54A32D192ED03ull ^ (idx + 1) * 0x8CB92BA72F3D8DD7ull ^ tag * 0xA0761D6478BD642Full;
    (void)rng_next(&r);
    return r;
}

/* uniform in [0, 1) with 53 random bits */
static double rng_u01(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* standard normal (Box-Muller, the cosine branch) */
static double rng_normal(rng_t *r)
{
    double u1 = rng_u01(r), u2 = rng_u01(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Poisson(lambda) by inversion of its cumulative distribution */
static int64_t rng_poisson(rng_t *r, double lambda)
{
    double u = rng_u01(r), p = exp(-lambda), c = p;
    int64_t k = 0;
    while (u > c && k < 100000) {
        ++k;
        p *= lambda / (double)k;
        c += p;
        if (p == 0.0 && c < u) break;
    }
    return k;
}

/* first index with cdf[idx] > u (cdf increasing, cdf[n - 1] = 1) */
static int64_t upper_index(const double *cdf, int64_t n, double u)
{
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* ------------------------------------------------------------------------ */
/* rows of X                                                                 */
/* ------------------------------------------------------------------------ */
#define ROW_TAG 0x524F5753ull   /* "ROWS" */

/* counts[i] = nonzeros of row i: Poisson(mean) clipped to [1, max(1, d / 2)] */
int synth_row_counts(int64_t n, int64_t d, double mean, uint64_t seed, int64_t *counts, int32_t nthreads)
{
    if (n < 0 || d <= 0 || !(mean > 0.0)) return -2;
    int64_t cmax = d / 2 > 1 ? d / 2 : 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(static, 4096)
    for (int64_t i = 0; i < n; ++i) {
        rng_t r = rng_stream(seed, (uint64_t)i, ROW_TAG);
        int64_t c = rng_poisson(&r, mean);
        counts[i] = c < 1 ? 1 : (c > cmax ? cmax : c);
    }
    return 0;
}

/*
 * Fills the rows of X (row_ptr from the counts above): each row's features
 * are distinct draws from the popularity law `cdf` over popularity ranks
 * (cdf[d - 1] = 1), mapped to feature ids by `perm`, sorted; values 1
 * (values_mode 0) or counts 1..8 from the truncated geometric law `vcdf`
 * (values_mode 1, vcdf[7] = 1).  The row's stream continues after its count.
 */
int synth_fill_rows(int64_t n, int64_t d, const double *cdf, const int64_t *perm, int32_t values_mode,
                    const double *vcdf, uint64_t seed, const int64_t *rp, int32_t *col, double *val,
                    int32_t nthreads)
{
    if (n < 0 || d <= 0) return -2;
    int failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        rng_t r = rng_stream(seed, (uint64_t)i, ROW_TAG);
        (void)rng_u01(&r);                     /* the draw of the row's count */
        int64_t c = rp[i + 1] - rp[i], have = 0, tries = 0;
        int32_t *row = col + rp[i];
        while (have < c) {
            if (++tries > 1000 * (c + 16)) {   /* cannot happen for c <= d / 2 */
#pragma omp atomic write
                failed = 1;
                break;
            }
            int64_t rank = upper_index(cdf, d, rng_u01(&r));
            int32_t f = (int32_t)perm[rank];
            /* insertion into the sorted row, skipping a repeated feature */
            int64_t lo = 0, hi = have;
            while (lo < hi) {
                int64_t mid = (lo + hi) / 2;
                if (row[mid] < f) lo = mid + 1; else hi = mid;
            }
            if (lo < have && row[lo] == f) continue;
            memmove(row + lo + 1, row + lo, (size_t)(have - lo) * sizeof(int32_t));
            row[lo] = f;
            ++have;
        }
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            val[e] = values_mode == 0 ? 1.0 : (double)(upper_index(vcdf, 8, rng_u01(&r)) + 1);
    }
    return failed ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* planted targets                                                           */
/* ------------------------------------------------------------------------ */
#define TGT_TAG 0x54475453ull   /* "TGTS" */

typedef struct { double s; int64_t i; } scored_t;

static int by_score_desc(const void *a, const void *b)
{
    const scored_t *x = (const scored_t *)a, *y = (const scored_t *)b;
    if (x->s > y->s) return -1;
    if (x->s < y->s) return 1;
    return x->i < y->i ? -1 : (x->i > y->i ? 1 : 0);
}

/*
 * T binary targets over the rows of X (CSR rp, col, val; n rows, d features).
 * Target t draws, from its own stream: n_inf informative features without
 * replacement from `pool` (npool feature ids), Gaussian weights w*; ell[t]
 * labelled rows and h_t = min(#unlabelled, max(1, ceil(holdout * ell[t])))
 * held-out rows, without replacement; the score z = x . w* plus Gaussian noise
 * of half z's standard deviation over those rows.  The n_pos = clip(round(q[t]
 * ell[t]), 1, ell[t] - 1) best-scored labelled rows are positive, the rest
 * negative; a held-out row's true class is its score against the midpoint of
 * the lowest positive and the highest negative score.
 *
 * labels[t][i]: +1 / -1 on the labelled rows, 0 elsewhere (the caller zeroes
 * it); truth[t][i]: the class of the labelled and held-out rows, 0 elsewhere;
 * held[t][0 .. h_t) (row ids, ascending) and nheld[t].  hmax bounds h_t.
 */
int synth_planted(int64_t n, int64_t d, const int64_t *rp, const int32_t *col, const double *val, int32_t T,
                  const int64_t *ell, const double *q, const int32_t *pool, int64_t npool, int64_t n_inf,
                  double holdout, uint64_t seed, int8_t *labels, int8_t *truth, int64_t *held, int64_t hmax,
                  int64_t *nheld, int32_t nthreads)
{
    if (n < 2 || d <= 0 || T < 0 || npool < n_inf || n_inf < 1) return -2;
    int failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double *wd = (double *)calloc((size_t)d, sizeof(double));      /* w* as a dense vector */
        unsigned char *mark = (unsigned char *)calloc((size_t)(n > npool ? n : npool), 1);
        int64_t *rows = (int64_t *)malloc((size_t)n * sizeof(int64_t));
        int32_t *inf = (int32_t *)malloc((size_t)n_inf * sizeof(int32_t));
        scored_t *sc = (scored_t *)malloc((size_t)n * sizeof(scored_t));
        double *z = (double *)malloc((size_t)n * sizeof(double));
        if (!wd || !mark || !rows || !inf || !sc || !z) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int32_t t = 0; t < T; ++t) {
                rng_t r = rng_stream(seed, (uint64_t)t, TGT_TAG);
                int8_t *lab = labels + (int64_t)t * n, *tru = truth + (int64_t)t * n;
                /* informative features and their weights */
                for (int64_t k = 0; k < n_inf;) {
                    int64_t j = (int64_t)(rng_u01(&r) * (double)npool);
                    if (j >= npool) j = npool - 1;
                    if (mark[j]) continue;
                    mark[j] = 1;
                    inf[k++] = (int32_t)j;
                }
                for (int64_t k = 0; k < n_inf; ++k) {
                    mark[inf[k]] = 0;
                    wd[pool[inf[k]]] = rng_normal(&r);
                }
                /* labelled rows, then held-out rows among the others */
                int64_t l = ell[t] < 2 ? 2 : (ell[t] > n ? n : ell[t]);
                int64_t h = (int64_t)ceil(holdout * (double)l);
                if (h < 1) h = 1;
                if (h > n - l) h = n - l;
                if (h > hmax) h = hmax;
                int64_t m = 0;
                while (m < l + h) {
                    int64_t i = (int64_t)(rng_u01(&r) * (double)n);
                    if (i >= n) i = n - 1;
                    if (mark[i]) continue;
                    mark[i] = 1;
                    rows[m++] = i;
                }
                /* scores of those rows and their spread */
                double s1 = 0.0, s2 = 0.0;
                for (int64_t k = 0; k < m; ++k) {
                    int64_t i = rows[k];
                    double zi = 0.0;
                    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) zi += val[e] * wd[col[e]];
                    z[k] = zi;
                    s1 += zi;
                    s2 += zi * zi;
                }
                double mean = s1 / (double)m, var = s2 / (double)m - mean * mean;
                double sd = var > 0.0 ? sqrt(var) : 1.0;
                for (int64_t k = 0; k < m; ++k) z[k] += 0.5 * sd * rng_normal(&r);
                /* classes of the labelled rows */
                for (int64_t k = 0; k < l; ++k) { sc[k].s = z[k]; sc[k].i = rows[k]; }
                qsort(sc, (size_t)l, sizeof(scored_t), by_score_desc);
                int64_t npos = (int64_t)llround(q[t] * (double)l);
                if (npos < 1) npos = 1;
                if (npos > l - 1) npos = l - 1;
                for (int64_t k = 0; k < l; ++k) {
                    lab[sc[k].i] = k < npos ? 1 : -1;
                    tru[sc[k].i] = lab[sc[k].i];
                }
                double thresh = 0.5 * (sc[npos - 1].s + sc[npos].s);
                /* held-out rows: true class from the threshold, ascending row ids */
                for (int64_t k = l; k < m; ++k) tru[rows[k]] = z[k] > thresh ? 1 : -1;
                int64_t *hl = held + (int64_t)t * hmax;
                for (int64_t k = l; k < m; ++k) hl[k - l] = rows[k];
                for (int64_t a = 1; a < h; ++a) {            /* insertion sort (h is small) */
                    int64_t v = hl[a], b = a - 1;
                    while (b >= 0 && hl[b] > v) { hl[b + 1] = hl[b]; --b; }
                    hl[b + 1] = v;
                }
                nheld[t] = h;
                for (int64_t k = 0; k < m; ++k) mark[rows[k]] = 0;
                for (int64_t k = 0; k < n_inf; ++k) wd[pool[inf[k]]] = 0.0;
            }
        }
        free(wd); free(mark); free(rows); free(inf); free(sc); free(z);
    }
    return failed ? -1 : 0;
}
