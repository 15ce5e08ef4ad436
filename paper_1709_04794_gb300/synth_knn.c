/*
 * Input-generator helper: k-nearest-neighbour lists of the rows of a sparse
 * sample x feature matrix under the Jaccard (Tanimoto) similarity of their
 * binary supports.  The similarity graph S of Sec. 2.3-2.4 (undirected kNN
 * graph, Tanimoto on fingerprints in Sec. 5.1) is an *input* of the solver;
 * this file only builds it.  It holds none of the solver's arithmetic.
 *
 * Candidates of row i are the rows j != i that share at least one feature
 * whose column count is <= cap.  With cap >= n every shared feature counts,
 * and the lists are the exact kNN among rows with nonzero similarity.
 * Neighbours are ranked by (similarity descending, row index ascending);
 * similarity 0 never makes a neighbour.  Each row is handled independently,
 * so the output does not depend on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
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
