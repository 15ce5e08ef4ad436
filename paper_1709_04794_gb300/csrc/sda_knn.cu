// The similarity graph S of Sec. 2.4 built on the device from the samples X:
// s_ij = Tanimoto (Jaccard) similarity of the binary supports of rows i and j,
// |x_i and x_j| / |x_i or x_j| (Tanimoto on fingerprints, Sec. 5.1); the edge
// set is the union of every row's k nearest rows (undirected kNN graph,
// Sec. 2.4), optionally keeping only similarities >= a threshold (the
// threshold graph of Sec. 2.4; Tanimoto >= 0.4 in Sec. 5.2).  Candidates of row
// i are the rows that share a feature whose column count is <= cap (every shared
// feature when cap >= N: the exact kNN); neighbours rank by (similarity
// descending, row index ascending) and similarity 0 never makes an edge.
#include <limits.h>

#include <vector>

#include "sda_common.cuh"

namespace sda {

constexpr int kKnnMaxK = 32;       // neighbours per row (one warp lane each)
constexpr int kKnnMaxRow = 1024;   // features of a row kept in shared memory
constexpr int kKnnWarps = 8;       // rows in flight per block (one warp each)

// rows sorted, columns in range and strictly increasing within a row (bit 1),
// row pointers monotone (bit 2), a row longer than kKnnMaxRow (bit 4)
__global__ void k_knn_check(int64_t n, int64_t d, const int64_t *rp, const int32_t *col, int *err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = rp[i], b = rp[i + 1];
        if (b < a) {
            atomicOr(err, 2);
            continue;
        }
        if (b - a > kKnnMaxRow) atomicOr(err, 4);
        int32_t prev = -1;
        for (int64_t e = a; e < b; ++e) {
            const int32_t c = col[e];
            if (c < 0 || c >= d || c <= prev) atomicOr(err, 1);
            prev = c;
        }
    }
}

__global__ void k_knn_colcount(int64_t nnz, const int32_t *col, unsigned long long *cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[col[e]], 1ull);
}

// rows of every column (inverted lists; the order within a column is not used)
__global__ void k_knn_fill(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *cp,
                           unsigned long long *fill, int32_t *crow) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int32_t f = col[e];
            crow[cp[f] + (int64_t)atomicAdd(&fill[f], 1ull)] = (int32_t)i;
        }
}

// The k nearest rows of every row: one warp per row.  Its features go to shared
// memory; the lanes take the candidates of the row's qualifying features 32 at a
// time and each computes |x_i and x_j| by binary search of x_j's features in x_i's;
// the 32 proposals then merge, one after the other, into the warp's sorted top-k
// (lane l < k holds slot l), a row already held being skipped.
__global__ void __launch_bounds__(kKnnWarps * 32) k_knn_rows(int64_t n, const int64_t *__restrict__ rp,
                                                              const int32_t *__restrict__ col,
                                                              const int64_t *__restrict__ cp,
                                                              const int32_t *__restrict__ crow, int64_t cap, int k,
                                                              double thr, int32_t *__restrict__ nbr,
                                                              double *__restrict__ sim) {
    __shared__ int32_t srow[kKnnWarps][kKnnMaxRow];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    for (int64_t i = (int64_t)blockIdx.x * kKnnWarps + w; i < n; i += (int64_t)gridDim.x * kKnnWarps) {
        const int64_t r0 = rp[i];
        const int li = (int)(rp[i + 1] - r0);
        __syncwarp();
        for (int q = lane; q < li; q += 32) srow[w][q] = col[r0 + q];
        __syncwarp();
        double bs = -1.0;         // slot `lane`: (similarity, row), sorted descending
        int32_t bj = INT_MAX;
        for (int q = 0; q < li; ++q) {
            const int32_t f = srow[w][q];
            const int64_t c0 = cp[f], c1 = cp[f + 1];
            if (c1 - c0 > cap) continue;
            for (int64_t base = c0; base < c1; base += 32) {
                const int64_t idx = base + lane;
                const int32_t j = idx < c1 ? crow[idx] : -1;
                double s = -1.0;
                if (j >= 0 && j != (int32_t)i) {
                    const int64_t a = rp[j], b = rp[j + 1];
                    int inter = 0;
                    for (int64_t e = a; e < b; ++e) {
                        const int32_t g = col[e];
                        int lo = 0, hi = li;
                        while (lo < hi) {
                            const int m = (lo + hi) >> 1;
                            if (srow[w][m] < g) lo = m + 1;
                            else hi = m;
                        }
                        inter += (lo < li && srow[w][lo] == g) ? 1 : 0;
                    }
                    if (inter > 0) s = (double)inter / (double)(li + (int)(b - a) - inter);
                    if (s < thr) s = -1.0;
                }
                for (int p = 0; p < 32; ++p) {
                    const double ps = __shfl_sync(full, s, p);
                    const int32_t pj = __shfl_sync(full, j, p);
                    if (!(ps > 0.0)) continue;
                    if (__any_sync(full, lane < k && bj == pj)) continue;
                    const bool beats = lane < k && (ps > bs || (ps == bs && pj < bj));
                    const unsigned m = __ballot_sync(full, beats);
                    if (m == 0u) continue;
                    const int pos = __ffs((int)m) - 1;
                    const double us = __shfl_up_sync(full, bs, 1);
                    const int32_t uj = __shfl_up_sync(full, bj, 1);
                    if (lane > pos && lane < k) {
                        bs = us;
                        bj = uj;
                    }
                    if (lane == pos) {
                        bs = ps;
                        bj = pj;
                    }
                }
            }
        }
        if (lane < k) {
            nbr[i * k + lane] = bs > 0.0 ? bj : -1;
            sim[i * k + lane] = bs > 0.0 ? bs : 0.0;
        }
    }
}

// directed entries of the union: e < n k is (i, nbr[e]), e >= n k the reverse of
// e - n k; an empty slot gets row n (sorts last)
__global__ void k_knn_keys(int64_t n, int k, const int32_t *nbr, uint32_t *keys, uint32_t *vals, int by_row,
                           const uint32_t *order) {
    const int64_t m = 2 * n * (int64_t)k;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = order ? (int64_t)order[q] : q;
        const int64_t ee = e < n * k ? e : e - n * k;
        const int32_t j = nbr[ee];
        uint32_t row, colv;
        if (j < 0) {
            row = colv = (uint32_t)n;
        } else if (e < n * k) {
            row = (uint32_t)(ee / k);
            colv = (uint32_t)j;
        } else {
            row = (uint32_t)j;
            colv = (uint32_t)(ee / k);
        }
        keys[q] = by_row ? row : colv;
        vals[q] = (uint32_t)e;
    }
}

// after the sort by (row, column): keep[q] = 1 for the first entry of each pair
// (row < n); rows of the kept entries counted
__global__ void k_knn_unique(int64_t n, int k, const int32_t *nbr, const uint32_t *order, int64_t *keep,
                             unsigned long long *rowcnt) {
    const int64_t m = 2 * n * (int64_t)k;
    auto pair_of = [&](int64_t q, uint32_t &row, uint32_t &c) {
        const int64_t e = order[q];
        const int64_t ee = e < n * k ? e : e - n * k;
        const int32_t j = nbr[ee];
        if (j < 0) {
            row = c = (uint32_t)n;
        } else if (e < n * k) {
            row = (uint32_t)(ee / k);
            c = (uint32_t)j;
        } else {
            row = (uint32_t)j;
            c = (uint32_t)(ee / k);
        }
    };
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
        uint32_t r, c, pr = UINT_MAX, pc = UINT_MAX;
        pair_of(q, r, c);
        if (q > 0) pair_of(q - 1, pr, pc);
        const bool first = r < (uint32_t)n && !(pr == r && pc == c);
        keep[q] = first ? 1 : 0;
        if (first) atomicAdd(&rowcnt[r], 1ull);
    }
}

__global__ void k_knn_emit(int64_t n, int k, const int32_t *nbr, const double *sim, const uint32_t *order,
                           const int64_t *keep, const int64_t *pos, int32_t *col_out, double *val_out) {
    const int64_t m = 2 * n * (int64_t)k;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[q]) continue;
        const int64_t e = order[q];
        const int64_t ee = e < n * k ? e : e - n * k;
        col_out[pos[q]] = e < n * k ? nbr[ee] : (int32_t)(ee / k);
        val_out[pos[q]] = sim[ee];
    }
}

__global__ void k_knn_rowptr(int64_t n, const unsigned long long *rowcnt, int64_t *rp) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
        rp[i] = i < n ? (int64_t)rowcnt[i] : 0;
}

static int grid_k(int64_t work, int sms) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + kBlock - 1) / kBlock, (int64_t)sms * 16));
}

static int key_bits(uint64_t v) {
    int b = 1;
    while (b < 32 && (v >> b) != 0) ++b;
    return b;
}

}  // namespace sda

using namespace sda;

extern "C" SDA_API int sda_knn_graph(const sda_csr *X, int32_t k, int64_t cap, double threshold, int64_t *row_ptr,
                                     int32_t *col_out, double *val_out, int64_t capacity, int64_t *nnz_out,
                                     void *cuda_stream) {
    clear_error();
    if (!X || !row_ptr || !nnz_out || (capacity > 0 && (!col_out || !val_out)))
        return fail(SDA_ERR_INVALID_ARG, "NULL argument");
    if (k < 1 || k > kKnnMaxK) return fail(SDA_ERR_INVALID_ARG, "k must be in [1, %d]", kKnnMaxK);
    if (!(threshold >= 0.0 && threshold <= 1.0)) return fail(SDA_ERR_INVALID_ARG, "threshold must be in [0, 1]");
    if (cap < 1) return fail(SDA_ERR_INVALID_ARG, "cap must be >= 1");
    const int64_t n = X->n_rows, d = X->n_cols, nnz = X->nnz;
    if (n < 1 || d < 1 || nnz < 0 || n >= (int64_t)UINT32_MAX / 2 || 2 * n * (int64_t)k >= (int64_t)UINT32_MAX ||
        d > INT32_MAX)
        return fail(SDA_ERR_SHAPE, "sizes out of range for the kNN graph");
    if (!X->row_ptr || (nnz > 0 && !X->col_idx)) return fail(SDA_ERR_INVALID_ARG, "missing array");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int sms = device_sm_count();
    if (sms <= 0) return fail(SDA_ERR_CUDA, "no CUDA device");
    DevBuf<int64_t> rp, cp;
    DevBuf<int32_t> col, crow, nbr;
    DevBuf<double> sim;
    DevBuf<unsigned long long> cnt;
    DevBuf<int> err;
    SDA_TRY(rp.alloc((size_t)n + 1));
    SDA_TRY(col.alloc((size_t)std::max<int64_t>(nnz, 1)));
    const cudaMemcpyKind kind = X->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    SDA_CUDA(cudaMemcpyAsync(rp.p, X->row_ptr, ((size_t)n + 1) * sizeof(int64_t), kind, s));
    if (nnz > 0) SDA_CUDA(cudaMemcpyAsync(col.p, X->col_idx, (size_t)nnz * sizeof(int32_t), kind, s));
    int64_t ends[2] = {0, 0};
    SDA_CUDA(cudaMemcpyAsync(&ends[0], rp.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaMemcpyAsync(&ends[1], rp.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    if (ends[0] != 0 || ends[1] != nnz) return fail(SDA_ERR_INDEX, "row_ptr must start at 0 and end at nnz");
    SDA_TRY(err.alloc(1));
    SDA_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    k_knn_check<<<grid_k(n, sms), kBlock, 0, s>>>(n, d, rp.p, col.p, err.p);
    SDA_LAUNCHED();
    int herr = 0;
    SDA_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    if (herr & 3) return fail(SDA_ERR_INDEX, "X: row pointers not monotone or a column out of range / unsorted");
    if (herr & 4) return fail(SDA_ERR_UNSUPPORTED, "a row of X holds more than %d features", kKnnMaxRow);
    // inverted lists (columns' rows)
    SDA_TRY(cnt.alloc((size_t)d + 1));
    SDA_TRY(cp.alloc((size_t)d + 1));
    SDA_TRY(crow.alloc((size_t)std::max<int64_t>(nnz, 1)));
    SDA_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.bytes(), s));
    k_knn_colcount<<<grid_k(nnz, sms), kBlock, 0, s>>>(nnz, col.p, cnt.p);
    SDA_LAUNCHED();
    SDA_CUDA(cudaMemcpyAsync(cp.p, cnt.p, ((size_t)d + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    SDA_TRY(scan_exclusive_i64(cp.p, d + 1, s));
    SDA_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.bytes(), s));
    k_knn_fill<<<grid_k(n, sms), kBlock, 0, s>>>(n, rp.p, col.p, cp.p, cnt.p, crow.p);
    SDA_LAUNCHED();
    // every row's k nearest
    SDA_TRY(nbr.alloc((size_t)(n * k)));
    SDA_TRY(sim.alloc((size_t)(n * k)));
    const int rb = (int)std::max<int64_t>(1, std::min<int64_t>((n + kKnnWarps - 1) / kKnnWarps, (int64_t)sms * 8));
    k_knn_rows<<<rb, kKnnWarps * 32, 0, s>>>(n, rp.p, col.p, cp.p, crow.p, cap, k, threshold > 0.0 ? threshold : 0.0,
                                             nbr.p, sim.p);
    SDA_LAUNCHED();
    // the union of the directed lists: entries sorted by (row, column), duplicates dropped
    const int64_t m = 2 * n * (int64_t)k;
    DevBuf<uint32_t> keys, vals;
    DevBuf<int64_t> keep, pos;
    SDA_TRY(keys.alloc((size_t)m));
    SDA_TRY(vals.alloc((size_t)m));
    k_knn_keys<<<grid_k(m, sms), kBlock, 0, s>>>(n, k, nbr.p, keys.p, vals.p, 0, nullptr);
    SDA_LAUNCHED();
    const int bits = key_bits((uint64_t)n);
    SDA_TRY(radix_sort_pairs(keys.p, vals.p, m, bits, s));
    DevBuf<uint32_t> order;
    SDA_TRY(order.alloc((size_t)m));
    SDA_CUDA(cudaMemcpyAsync(order.p, vals.p, (size_t)m * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    k_knn_keys<<<grid_k(m, sms), kBlock, 0, s>>>(n, k, nbr.p, keys.p, vals.p, 1, order.p);
    SDA_LAUNCHED();
    SDA_TRY(radix_sort_pairs(keys.p, vals.p, m, bits, s));
    SDA_TRY(keep.alloc((size_t)m + 1));
    SDA_TRY(pos.alloc((size_t)m + 1));
    DevBuf<unsigned long long> rowcnt;
    SDA_TRY(rowcnt.alloc((size_t)n + 1));
    SDA_CUDA(cudaMemsetAsync(rowcnt.p, 0, rowcnt.bytes(), s));
    k_knn_unique<<<grid_k(m, sms), kBlock, 0, s>>>(n, k, nbr.p, vals.p, keep.p, rowcnt.p);
    SDA_LAUNCHED();
    SDA_CUDA(cudaMemsetAsync(keep.p + m, 0, sizeof(int64_t), s));
    SDA_CUDA(cudaMemcpyAsync(pos.p, keep.p, ((size_t)m + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    SDA_TRY(scan_exclusive_i64(pos.p, m + 1, s));
    int64_t total = 0;
    SDA_CUDA(cudaMemcpyAsync(&total, pos.p + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    *nnz_out = total;
    if (total > capacity)
        return fail(SDA_ERR_SHAPE, "the graph has %lld entries, the output holds %lld", (long long)total,
                    (long long)capacity);
    k_knn_emit<<<grid_k(m, sms), kBlock, 0, s>>>(n, k, nbr.p, sim.p, vals.p, keep.p, pos.p, col_out, val_out);
    SDA_LAUNCHED();
    k_knn_rowptr<<<grid_k(n + 1, sms), kBlock, 0, s>>>(n, rowcnt.p, row_ptr);
    SDA_LAUNCHED();
    SDA_TRY(scan_exclusive_i64(row_ptr, n + 1, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    return SDA_OK;
}
