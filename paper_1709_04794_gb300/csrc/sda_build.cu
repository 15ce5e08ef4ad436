// sda_build_operator: everything the solves of one (X, S, labels) share.
//
//  - X is validated, its features relabelled by descending column count
//    (stable in the feature id), and stored twice in the compute dtype: CSR
//    with the new column ids and CSC (new column order, rows ascending), the
//    CSC built by a stable radix sort of the nonzeros by column.
//  - S is validated (CSR, weights >= 0) and checked to equal its transpose;
//    the degrees D_ii = sum_j s_ij of L = D - S (Sec. 2.3) are formed.
//  - For every target: l, N+, N-, and from the exact column sums
//    X^T 1_+ and X^T 1_- (Alg. 7 step 3): mu_l = (X^T 1_+ + X^T 1_-) / l and
//    d = X^T 1_+ / N+ - X^T 1_- / N-.
#include <math.h>

#include <algorithm>
#include <vector>

#include "sda_kernels.cuh"

namespace sda {

enum : int {
    kErrIndex = 1,
    kErrInexact = 2,
    kErrNonFinite = 4,
    kErrWeight = 8,
    kErrAsym = 16,
    kErrLabel = 32,
    kErrRowPtr = 64,
};

// ---------------------------------------------------------------------------
// conversions
// ---------------------------------------------------------------------------
template <class T>
struct Store;
template <>
struct Store<double> {
    static __device__ __forceinline__ double make(double x) { return x; }
    static __device__ __forceinline__ double back(double x) { return x; }
};
template <>
struct Store<float> {
    static __device__ __forceinline__ float make(double x) { return (float)x; }
    static __device__ __forceinline__ double back(float x) { return (double)x; }
};
template <>
struct Store<__half> {
    static __device__ __forceinline__ __half make(double x) { return __double2half(x); }
    static __device__ __forceinline__ double back(__half x) { return (double)__half2float(x); }
};
template <>
struct Store<__nv_fp8_e4m3> {
    static __device__ __forceinline__ __nv_fp8_e4m3 make(double x) { return __nv_fp8_e4m3((float)x); }
    static __device__ __forceinline__ double back(__nv_fp8_e4m3 x) { return (double)float(x); }
};

__device__ __forceinline__ double load_in(const void *v, int dtype, int64_t e) {
    if (dtype == SDA_F64) return ((const double *)v)[e];
    if (dtype == SDA_F32) return (double)((const float *)v)[e];
    return 1.0;
}

// ---------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------
__global__ void k_check_csr(int64_t n, int64_t ncols, const int64_t *rp, const int32_t *col, const void *val,
                            int dtype, int nonneg, int *err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = rp[i], b = rp[i + 1];
        if (b < a) {
            atomicOr(err, kErrRowPtr);
            continue;
        }
        int32_t prev = -1;
        for (int64_t e = a; e < b; ++e) {
            const int32_t c = col[e];
            if (c < 0 || c >= ncols || c <= prev) atomicOr(err, kErrIndex);
            prev = c;
            if (val) {
                const double x = load_in(val, dtype, e);
                if (!isfinite(x)) atomicOr(err, kErrNonFinite);
                if (nonneg && x < 0.0) atomicOr(err, kErrWeight);
            }
        }
    }
}

__global__ void k_col_count(int64_t nnz, const int32_t *col, unsigned long long *cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[col[e]], 1ull);
}

__global__ void k_perm_keys(int64_t d, const unsigned long long *cnt, unsigned long long maxc, uint32_t *keys,
                            uint32_t *vals) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x) {
        keys[j] = (uint32_t)(maxc - cnt[j]);
        vals[j] = (uint32_t)j;
    }
}

__global__ void k_perm_finish(int64_t d, const uint32_t *old_sorted, const unsigned long long *cnt,
                              int32_t *old_of_new, int32_t *new_of_old, int64_t *cp) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < d; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = (int32_t)old_sorted[k];
        old_of_new[k] = o;
        new_of_old[o] = (int32_t)k;
        cp[k] = (int64_t)cnt[o];
    }
}

__global__ void k_relabel(int64_t nnz, const int32_t *col_in, const int32_t *new_of_old, int32_t *col_out,
                          uint32_t *keys, uint32_t *vals) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = new_of_old ? new_of_old[col_in[e]] : col_in[e];
        col_out[e] = c;
        keys[e] = (uint32_t)c;
        vals[e] = (uint32_t)e;
    }
}

__global__ void k_expand_rows(int64_t n, const int64_t *rp, int32_t *row_of) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) row_of[e] = (int32_t)i;
}

__global__ void k_gather_rows(int64_t nnz, const uint32_t *src, const int32_t *row_of, int32_t *out) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = row_of[src[k]];
}

// out[k] = store(in[src ? src[k] : k]); flags values that do not survive the round trip
template <class OUT>
__global__ void k_convert(int64_t m, const void *in, int dtype, const uint32_t *src, OUT *out, int *err) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = src ? (int64_t)src[k] : k;
        const double x = load_in(in, dtype, e);
        const OUT y = Store<OUT>::make(x);
        if (Store<OUT>::back(y) != x) atomicOr(err, kErrInexact);
        out[k] = y;
    }
}

// pattern storage: every value must be exactly one
__global__ void k_check_ones(int64_t m, const void *in, int dtype, int *err) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        if (load_in(in, dtype, k) != 1.0) atomicOr(err, kErrInexact);
}

// S == S^T: the k-th nonzero of S^T (sorted by column of S, stable) must match the k-th of S
__global__ void k_check_sym(int64_t nnz, const uint32_t *tkey, const uint32_t *tsrc, const int32_t *row_of,
                            const int32_t *col, const void *val, int dtype, int *err) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = tsrc[k];
        const bool same = ((int32_t)tkey[k] == row_of[k]) && (row_of[e] == col[k]) &&
                          (!val || load_in(val, dtype, e) == load_in(val, dtype, k));
        if (!same) atomicOr(err, kErrAsym);
    }
}

// degrees from the stored weights (FP64 sums), FP64 and vector-type copies
template <class FT>
__global__ void k_degrees(int64_t n, const int64_t *rp, const void *val, int dtype, double *s64, FT *sft,
                          double *deg64, FT *degft) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0, sf = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const double x = load_in(val, dtype, e);
            s64[e] = x;
            if (sft) {
                const FT xf = (FT)x;
                sft[e] = xf;
                sf += (double)xf;
            }
            s += x;
        }
        deg64[i] = s;
        if (degft) degft[i] = (FT)sf;
    }
}

__global__ void k_check_labels(int64_t m, const int8_t *y, int *err) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        if (y[k] < -1 || y[k] > 1) atomicOr(err, kErrLabel);
}

__global__ void k_indicators(int64_t n, const int8_t *y, double *ip, double *in_, unsigned long long *cnt) {
    unsigned long long cp = 0, cn = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        ip[i] = y[i] > 0 ? 1.0 : 0.0;
        in_[i] = y[i] < 0 ? 1.0 : 0.0;
        cp += y[i] > 0;
        cn += y[i] < 0;
    }
    cp = warp_sum(cp);
    cn = warp_sum(cn);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&cnt[0], cp);
        atomicAdd(&cnt[1], cn);
    }
}

__global__ void k_means(int64_t d, const double *sp, const double *sn, double npos, double nneg, double *mu,
                        float *mu32, double *dv) {
    const double ell = npos + nneg;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x) {
        const double m = (sp[j] + sn[j]) / ell;
        mu[j] = m;
        mu32[j] = (float)m;
        dv[j] = sp[j] / npos - sn[j] / nneg;
    }
}

// ---- X split into ranges of rows (column pass of the iteration) ----------------
// lb[r][j] = first entry of column j whose row is at least r * rb (rows ascend
// within a column); cnt[r][j] = entries of column j in range r, cnt[r][d] = 0
__global__ void k_range_bounds(int64_t d, int nr, int64_t rb, const int64_t *cp, const int32_t *row, int64_t *lb,
                               int64_t *cnt) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = cp[j], hi = cp[j + 1];
        int64_t prev = lo;
        lb[j] = lo;
        for (int r = 1; r <= nr; ++r) {
            int64_t a = prev, b = hi;
            if (r == nr) {
                a = hi;
            } else {
                const int64_t bound = (int64_t)r * rb;
                while (a < b) {
                    const int64_t m = a + (b - a) / 2;
                    if ((int64_t)row[m] < bound) a = m + 1;
                    else b = m;
                }
            }
            lb[(int64_t)r * d + j] = a;
            cnt[(int64_t)(r - 1) * (d + 1) + j] = (a - prev + 3) / 4 * 4;   // padded to a quad
            prev = a;
        }
    }
}

// entry e of the CSC goes to range r = row / rb at xb_cp[r][j] + (e - lb[r][j]);
// the padding after each segment stays zero (row 0, value 0)
__global__ void k_range_scatter(int64_t nnz, int64_t d, int64_t rb, const int64_t *cp, const int32_t *row,
                                const char *val, int vsz, const int64_t *lb, const int64_t *xcp, uint16_t *xrow,
                                char *xval) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = 0, b = d;   // largest j with cp[j] <= e
        while (b - a > 1) {
            const int64_t m = a + (b - a) / 2;
            if (cp[m] <= e) a = m;
            else b = m;
        }
        const int64_t j = a, i = row[e], r = i / rb;
        const int64_t pos = xcp[r * (d + 1) + j] + (e - lb[r * d + j]);
        xrow[pos] = (uint16_t)(i - r * rb);
        switch (vsz) {
        case 0: xval[pos] = (char)0x38; break;   // pattern: an FP8 E4M3 one
        case 1: xval[pos] = val[e]; break;
        case 2: reinterpret_cast<uint16_t *>(xval)[pos] = reinterpret_cast<const uint16_t *>(val)[e]; break;
        case 4: reinterpret_cast<uint32_t *>(xval)[pos] = reinterpret_cast<const uint32_t *>(val)[e]; break;
        case 8:
            reinterpret_cast<unsigned long long *>(xval)[pos] = reinterpret_cast<const unsigned long long *>(val)[e];
            break;
        default: break;
        }
    }
}

// padded row lengths of X (quads)
__global__ void k_row_quads(int64_t n, const int64_t *rp, int64_t *cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        cnt[i] = (rp[i + 1] - rp[i] + 3) / 4 * 4;
}

// entry e of row i goes to xrp[i] + (e - rp[i]); the padding stays zero
__global__ void k_row_scatter(int64_t nnz, int64_t n, const int64_t *rp, const int32_t *col, const char *val, int vsz,
                              const int64_t *xrp, int32_t *xcol, char *xval) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = 0, b = n;   // largest i with rp[i] <= e
        while (b - a > 1) {
            const int64_t m = a + (b - a) / 2;
            if (rp[m] <= e) a = m;
            else b = m;
        }
        const int64_t pos = xrp[a] + (e - rp[a]);
        xcol[pos] = col[e];
        switch (vsz) {
        case 0: xval[pos] = (char)0x38; break;   // pattern: an FP8 E4M3 one
        case 1: xval[pos] = val[e]; break;
        case 2: reinterpret_cast<uint16_t *>(xval)[pos] = reinterpret_cast<const uint16_t *>(val)[e]; break;
        case 4: reinterpret_cast<uint32_t *>(xval)[pos] = reinterpret_cast<const uint32_t *>(val)[e]; break;
        case 8:
            reinterpret_cast<unsigned long long *>(xval)[pos] = reinterpret_cast<const unsigned long long *>(val)[e];
            break;
        default: break;
        }
    }
}

static int grid1(int64_t work, int sms) {
    int64_t g = (work + kBlock - 1) / kBlock;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)sms * 16));
}

static int bits_for(unsigned long long v) {
    int b = 0;
    while (b < 64 && (v >> b) != 0ull) ++b;
    return b;
}

static int read_err(DevBuf<int> &err, cudaStream_t s, int *host) {
    SDA_CUDA(cudaMemcpyAsync(host, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    return SDA_OK;
}

// copies a host or device array to a new device buffer
template <class T>
static int to_device(DevBuf<T> &dst, const void *src, int64_t count, int on_device, cudaStream_t s) {
    SDA_TRY(dst.alloc((size_t)std::max<int64_t>(count, 1)));
    if (count > 0)
        SDA_CUDA(cudaMemcpyAsync(dst.p, src, (size_t)count * sizeof(T),
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return SDA_OK;
}

static size_t dtype_size(int dt) {
    switch (dt) {
    case SDA_F64: return 8;
    case SDA_F32: return 4;
    case SDA_F16: return 2;
    case SDA_F8E4M3: return 1;
    default: return 0;
    }
}

template <class OUT>
static int convert(int64_t m, const void *in, int dtype, const uint32_t *src, void *out, int *err, int sms,
                   cudaStream_t s) {
    k_convert<OUT><<<grid1(m, sms), kBlock, 0, s>>>(m, in, dtype, src, (OUT *)out, err);
    SDA_LAUNCHED();
    return SDA_OK;
}

static int convert_any(int compute, int64_t m, const void *in, int dtype, const uint32_t *src, void *out, int *err,
                       int sms, cudaStream_t s) {
    switch (compute) {
    case SDA_F64: return convert<double>(m, in, dtype, src, out, err, sms, s);
    case SDA_F32: return convert<float>(m, in, dtype, src, out, err, sms, s);
    case SDA_F16: return convert<__half>(m, in, dtype, src, out, err, sms, s);
    case SDA_F8E4M3: return convert<__nv_fp8_e4m3>(m, in, dtype, src, out, err, sms, s);
    default: return fail(SDA_ERR_INVALID_ARG, "unknown compute dtype %d", compute);
    }
}

// lanes per row of the register row pass (four loads per lane per round): the
// 90th percentile of the row lengths fits one round
static int row_lanes(const std::vector<int64_t> &rp) {
    const int64_t n = (int64_t)rp.size() - 1;
    if (n <= 0) return 4;
    std::vector<int64_t> len((size_t)n);
    for (int64_t i = 0; i < n; ++i) len[(size_t)i] = rp[(size_t)i + 1] - rp[(size_t)i];
    const size_t k = (size_t)(0.9 * (double)(n - 1));
    std::nth_element(len.begin(), len.begin() + k, len.end());
    const int64_t p90 = len[k];
    int g = 4;
    while (g < 32 && 4 * g < p90) g <<= 1;
    return g;
}

// A matrix of nseg segments over nidx indices (CSC-like: ptr, idx, val) split
// into ranges of the index small enough that one range's slice of an nidx-vector
// of the iteration type fits a block's shared memory (at most 65280 indices:
// 16-bit local indices), equal in size up to a multiple of 256.  Each (range,
// segment) is padded with zero entries to a multiple of four (quads: one 8-byte
// load of indices per four entries); a pattern matrix (vsz 0) gets explicit FP8
// ones.  Indices ascend within each segment (the range bounds are found by
// binary search).
static int build_range_blocks(sda_operator *op, RangeBlocks &out, const int64_t *ptr, const int32_t *idx,
                              const char *val, size_t vsz, int64_t nseg, int64_t nidx, int64_t nnz, size_t fsz,
                              int sms, cudaStream_t s) {
    int optin = 0, per_sm = 0;
    SDA_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, op->device));
    SDA_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, op->device));
    const int64_t budget =
        std::min<int64_t>(optin, per_sm / kColBlkPerSm) - kColBlkReserve - colblk_scratch((int64_t)fsz);
    const int64_t rb_max = std::min<int64_t>(65280, budget / (int64_t)fsz / 256 * 256);
    if (rb_max < 256) return fail(SDA_ERR_UNSUPPORTED, "not enough shared memory per block for the range passes");
    const int64_t nr = std::max<int64_t>(1, (nidx + rb_max - 1) / rb_max);
    const int64_t rb = ((nidx + nr - 1) / nr + 255) / 256 * 256;
    out.nranges = (int)nr;
    out.rb = rb;
    out.nseg = nseg;
    SDA_TRY(out.cp.alloc((size_t)(nr * (nseg + 1))));
    SDA_CUDA(cudaMemsetAsync(out.cp.p, 0, out.cp.bytes(), s));
    DevBuf<int64_t> lb;
    SDA_TRY(lb.alloc((size_t)((nr + 1) * nseg)));
    k_range_bounds<<<grid1(nseg, sms), kBlock, 0, s>>>(nseg, (int)nr, rb, ptr, idx, lb.p, out.cp.p);
    SDA_LAUNCHED();
    SDA_TRY(scan_exclusive_i64(out.cp.p, nr * (nseg + 1), s));
    std::vector<int64_t> hp((size_t)(nr * (nseg + 1)));
    SDA_CUDA(cudaMemcpyAsync(hp.data(), out.cp.p, hp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    const int64_t nq = std::max<int64_t>(hp.back(), 4);   // padded entries
    const size_t bvsz = vsz ? vsz : 1;
    SDA_TRY(out.idx.alloc((size_t)nq));
    SDA_TRY(out.val.alloc((size_t)nq * bvsz));
    SDA_CUDA(cudaMemsetAsync(out.idx.p, 0, out.idx.bytes(), s));
    SDA_CUDA(cudaMemsetAsync(out.val.p, 0, out.val.bytes(), s));
    k_range_scatter<<<grid1(nnz, sms), kBlock, 0, s>>>(nnz, nseg, rb, ptr, idx, val, (int)vsz, lb.p, out.cp.p,
                                                       out.idx.p, out.val.p);
    SDA_LAUNCHED();
    std::vector<int32_t> off;
    out.per_range = std::max(1, sms * kColBlkPerSm / (int)nr);
    SDA_TRY(build_range_schedule(hp, (int)nr, nseg, out.sched, off, warp_chunk_nnz((int64_t)fsz)));
    SDA_TRY(out.tile_off.alloc(off.size()));
    SDA_CUDA(cudaMemcpy(out.tile_off.p, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    return SDA_OK;
}

// The head columns of X (the most frequent features: the fewest covering
// kHeadCover of the nonzeros, at most kHeadMax, each with at least one entry
// per range on average) split into ranges of kHeadRows rows with 16-bit local
// row indices, for the batched column pass: a block keeps one range's slice of
// the 16 targets' vectors in shared memory and gathers from it.
static int build_head_blocks(sda_operator *op, const char *val, size_t vsz, int64_t n, int64_t d, int sms,
                             cudaStream_t s) {
    RangeBlocks &out = op->hb;
    const int64_t nr = (n + kHeadRows - 1) / kHeadRows;
    std::vector<int64_t> cp((size_t)std::min<int64_t>(d, kHeadMax) + 1);
    SDA_CUDA(cudaMemcpyAsync(cp.data(), op->x_cp.p, cp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    int64_t nnz_all = 0;
    SDA_CUDA(cudaMemcpyAsync(&nnz_all, op->x_cp.p + d, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    int64_t h = 0;
    while (h < (int64_t)cp.size() - 1 && cp[(size_t)h] < kHeadCover * (double)nnz_all &&
           cp[(size_t)h + 1] - cp[(size_t)h] >= nr)
        ++h;
    out.nranges = (int)nr;
    out.rb = kHeadRows;
    out.nseg = h;
    if (h == 0) return SDA_OK;
    const int64_t nnz_h = cp[(size_t)h];
    SDA_TRY(out.cp.alloc((size_t)(nr * (h + 1))));
    SDA_CUDA(cudaMemsetAsync(out.cp.p, 0, out.cp.bytes(), s));
    DevBuf<int64_t> lb;
    SDA_TRY(lb.alloc((size_t)((nr + 1) * h)));
    k_range_bounds<<<grid1(h, sms), kBlock, 0, s>>>(h, (int)nr, kHeadRows, op->x_cp.p, op->x_row.p, lb.p, out.cp.p);
    SDA_LAUNCHED();
    SDA_TRY(scan_exclusive_i64(out.cp.p, nr * (h + 1), s));
    int64_t nq = 0;
    SDA_CUDA(cudaMemcpyAsync(&nq, out.cp.p + nr * (h + 1) - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    nq = std::max<int64_t>(nq, 4);
    const size_t bvsz = vsz ? vsz : 1;
    SDA_TRY(out.idx.alloc((size_t)nq));
    SDA_TRY(out.val.alloc((size_t)nq * bvsz));
    SDA_CUDA(cudaMemsetAsync(out.idx.p, 0, out.idx.bytes(), s));
    SDA_CUDA(cudaMemsetAsync(out.val.p, 0, out.val.bytes(), s));
    k_range_scatter<<<grid1(nnz_h, sms), kBlock, 0, s>>>(nnz_h, h, kHeadRows, op->x_cp.p, op->x_row.p, val,
                                                         (int)vsz, lb.p, out.cp.p, out.idx.p, out.val.p);
    SDA_LAUNCHED();
    return SDA_OK;
}

// Rows of X padded to whole quads for the row pass of the iteration, and the
// number of leading (most frequent) features it keeps in shared memory.
static int build_row_quads(sda_operator *op, bool fp64, size_t vsz, int sms, cudaStream_t s) {
    const int64_t n = op->n, d = op->d, nnz = op->nnz;
    SDA_TRY(op->xr_rp.alloc((size_t)n + 1));
    SDA_CUDA(cudaMemsetAsync(op->xr_rp.p + n, 0, sizeof(int64_t), s));
    k_row_quads<<<grid1(n, sms), kBlock, 0, s>>>(n, op->x_rp.p, op->xr_rp.p);
    SDA_LAUNCHED();
    SDA_TRY(scan_exclusive_i64(op->xr_rp.p, n + 1, s));
    std::vector<int64_t> hp((size_t)n + 1);
    SDA_CUDA(cudaMemcpyAsync(hp.data(), op->xr_rp.p, hp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    const int64_t nq = std::max<int64_t>(hp.back(), 4);
    const size_t bvsz = vsz ? vsz : 1;
    SDA_TRY(op->xr_col.alloc((size_t)nq));
    SDA_TRY(op->xr_val.alloc((size_t)nq * bvsz));
    SDA_CUDA(cudaMemsetAsync(op->xr_col.p, 0, op->xr_col.bytes(), s));
    SDA_CUDA(cudaMemsetAsync(op->xr_val.p, 0, op->xr_val.bytes(), s));
    k_row_scatter<<<grid1(nnz, sms), kBlock, 0, s>>>(nnz, n, op->x_rp.p, op->x_col.p, op->x_val_r.p, (int)vsz,
                                                     op->xr_rp.p, op->xr_col.p, op->xr_val.p);
    SDA_LAUNCHED();
    // lanes per row: the fewest (2..32) whose two quads per lane cover the median row
    std::vector<int64_t> len((size_t)n);
    for (int64_t i = 0; i < n; ++i) len[(size_t)i] = hp[(size_t)i + 1] - hp[(size_t)i];
    int64_t med = 0;
    if (n > 0) {
        std::nth_element(len.begin(), len.begin() + n / 2, len.end());
        med = len[(size_t)(n / 2)];
    }
    int g = 2;
    while (g < 32 && 8 * g < med) g <<= 1;
    op->xr_lanes = g;
    // head of p kept in shared memory: the fewest leading (most frequent) features
    // that hold kRowHeadCover of the nonzeros, at most kRowHeadMax and what a
    // block's shared memory allows (every block forms the head once per
    // iteration, so a larger head costs more than its extra gathers save)
    int optin = 0, per_sm = 0;
    SDA_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, op->device));
    SDA_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, op->device));
    const int64_t fsz = fp64 ? 8 : 4;
    const int64_t budget = std::min<int64_t>(optin, per_sm / kColBlkPerSm) - kColBlkReserve;
    const int64_t hmax = std::min<int64_t>(kRowHeadMax, std::max<int64_t>(0, budget / fsz / 256 * 256));
    std::vector<int64_t> cp((size_t)d + 1);
    SDA_CUDA(cudaMemcpy(cp.data(), op->x_cp.p, cp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
    const int64_t goal = (int64_t)std::ceil(kRowHeadCover * (double)nnz);
    const int64_t cover = std::lower_bound(cp.begin(), cp.end(), goal) - cp.begin();
    const int64_t head = (cover + 255) / 256 * 256;
    op->xr_head = (int)std::min(std::min<int64_t>(hmax, head), d / 8 * 8);   // whole 16-byte vectors of pairs
    return SDA_OK;
}

static int build(const sda_csr *X, const sda_csr *S, const sda_labels *y, double alpha, double omega,
                 sda_dtype compute, cudaStream_t s, sda_operator *op) {
    const int64_t n = X->n_rows, d = X->n_cols, nnz = X->nnz, snz = S->nnz;
    const int sms = op->sm_count;
    const int x_in_dt = X->values ? X->dtype : SDA_PATTERN;
    const int s_in_dt = S->values ? S->dtype : SDA_PATTERN;
    const bool fp64 = compute == SDA_F64;
    int herr = 0;
    DevBuf<int> err;
    SDA_TRY(err.alloc(1));
    SDA_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));

    // ---- X: copy and validate ----------------------------------------------
    DevBuf<int32_t> col_in;
    DevBuf<char> val_in;
    SDA_TRY(to_device(op->x_rp, X->row_ptr, n + 1, X->on_device, s));
    SDA_TRY(to_device(col_in, X->col_idx, nnz, X->on_device, s));
    if (X->values) {
        const size_t vb = dtype_size(X->dtype);
        SDA_TRY(val_in.alloc((size_t)std::max<int64_t>(nnz, 1) * vb));
        if (nnz > 0)
            SDA_CUDA(cudaMemcpyAsync(val_in.p, X->values, (size_t)nnz * vb,
                                     X->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    }
    int64_t ends[2];
    SDA_CUDA(cudaMemcpyAsync(&ends[0], op->x_rp.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaMemcpyAsync(&ends[1], op->x_rp.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    if (ends[0] != 0 || ends[1] != nnz)
        return fail(SDA_ERR_INDEX, "X row_ptr must start at 0 and end at nnz (got %lld .. %lld, nnz %lld)",
                    (long long)ends[0], (long long)ends[1], (long long)nnz);
    k_check_csr<<<grid1(n, sms), kBlock, 0, s>>>(n, d, op->x_rp.p, col_in.p, X->values ? val_in.p : nullptr,
                                                 x_in_dt, 0, err.p);
    SDA_LAUNCHED();
    SDA_TRY(read_err(err, s, &herr));
    if (herr & (kErrIndex | kErrRowPtr))
        return fail(SDA_ERR_INDEX, "X: row pointers not monotone or a column index out of range / not strictly "
                                   "increasing within its row");
    if (herr & kErrNonFinite) return fail(SDA_ERR_VALUE_NOT_EXACT, "X holds a non-finite value");

    // ---- feature order by descending column count ---------------------------
    DevBuf<unsigned long long> cnt;
    SDA_TRY(cnt.alloc((size_t)std::max<int64_t>(d, 1)));
    SDA_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)d * sizeof(unsigned long long), s));
    k_col_count<<<grid1(nnz, sms), kBlock, 0, s>>>(nnz, col_in.p, cnt.p);
    SDA_LAUNCHED();
    std::vector<unsigned long long> hcnt((size_t)d);
    SDA_CUDA(cudaMemcpyAsync(hcnt.data(), cnt.p, (size_t)d * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    unsigned long long maxc = 0;
    for (auto c : hcnt) maxc = std::max(maxc, c);
    SDA_TRY(op->new_of_old.alloc((size_t)d));
    SDA_TRY(op->old_of_new.alloc((size_t)d));
    SDA_TRY(op->x_cp.alloc((size_t)d + 1));
    {
        DevBuf<uint32_t> keys, vals;
        SDA_TRY(keys.alloc((size_t)d));
        SDA_TRY(vals.alloc((size_t)d));
        k_perm_keys<<<grid1(d, sms), kBlock, 0, s>>>(d, cnt.p, maxc, keys.p, vals.p);
        SDA_LAUNCHED();
        SDA_TRY(radix_sort_pairs(keys.p, vals.p, d, bits_for(maxc), s));
        k_perm_finish<<<grid1(d, sms), kBlock, 0, s>>>(d, vals.p, cnt.p, op->old_of_new.p, op->new_of_old.p,
                                                       op->x_cp.p);
        SDA_LAUNCHED();
        SDA_CUDA(cudaMemsetAsync(op->x_cp.p + d, 0, sizeof(int64_t), s));
        SDA_TRY(scan_exclusive_i64(op->x_cp.p, d + 1, s));
    }

    // ---- CSR with new column ids, CSC by stable sort on the column ------------
    SDA_TRY(op->x_col.alloc((size_t)std::max<int64_t>(nnz, 1)));
    SDA_TRY(op->x_row.alloc((size_t)std::max<int64_t>(nnz, 1)));
    const size_t vsz = compute == SDA_PATTERN ? 0 : dtype_size(compute);
    if (vsz) {
        SDA_TRY(op->x_val_r.alloc((size_t)std::max<int64_t>(nnz, 1) * vsz));
        SDA_TRY(op->x_val_c.alloc((size_t)std::max<int64_t>(nnz, 1) * vsz));
    }
    {
        DevBuf<uint32_t> keys, vals;
        DevBuf<int32_t> row_of;
        SDA_TRY(keys.alloc((size_t)std::max<int64_t>(nnz, 1)));
        SDA_TRY(vals.alloc((size_t)std::max<int64_t>(nnz, 1)));
        SDA_TRY(row_of.alloc((size_t)std::max<int64_t>(nnz, 1)));
        k_relabel<<<grid1(nnz, sms), kBlock, 0, s>>>(nnz, col_in.p, op->new_of_old.p, op->x_col.p, keys.p, vals.p);
        SDA_LAUNCHED();
        SDA_TRY(radix_sort_pairs(keys.p, vals.p, nnz, bits_for((unsigned long long)std::max<int64_t>(d - 1, 1)), s));
        k_expand_rows<<<grid1(n, sms), kBlock, 0, s>>>(n, op->x_rp.p, row_of.p);
        SDA_LAUNCHED();
        k_gather_rows<<<grid1(nnz, sms), kBlock, 0, s>>>(nnz, vals.p, row_of.p, op->x_row.p);
        SDA_LAUNCHED();
        if (vsz) {
            SDA_TRY(convert_any(compute, nnz, X->values ? (const void *)val_in.p : nullptr, x_in_dt, nullptr,
                                op->x_val_r.p, err.p, sms, s));
            SDA_TRY(convert_any(compute, nnz, X->values ? (const void *)val_in.p : nullptr, x_in_dt, vals.p,
                                op->x_val_c.p, err.p, sms, s));
        } else if (X->values) {
            k_check_ones<<<grid1(nnz, sms), kBlock, 0, s>>>(nnz, val_in.p, x_in_dt, err.p);
            SDA_LAUNCHED();
        }
        SDA_TRY(read_err(err, s, &herr));
        if (herr & kErrInexact)
            return fail(SDA_ERR_VALUE_NOT_EXACT, "a value of X is not exact in the compute dtype %d", (int)compute);
    }
    SDA_TRY(build_range_blocks(op, op->xb, op->x_cp.p, op->x_row.p, op->x_val_c.p, vsz, d, n, nnz,
                               fp64 ? sizeof(double) : sizeof(float), sms, s));
    SDA_TRY(build_row_quads(op, fp64, vsz, sms, s));
    SDA_TRY(build_head_blocks(op, op->x_val_c.p, vsz, n, d, sms, s));

    // ---- S -------------------------------------------------------------------
    DevBuf<int32_t> s_col_in;
    DevBuf<char> s_val_in;
    SDA_TRY(to_device(op->s_rp, S->row_ptr, n + 1, S->on_device, s));
    SDA_TRY(to_device(op->s_col, S->col_idx, snz, S->on_device, s));
    if (S->values) {
        const size_t vb = dtype_size(S->dtype);
        SDA_TRY(s_val_in.alloc((size_t)std::max<int64_t>(snz, 1) * vb));
        if (snz > 0)
            SDA_CUDA(cudaMemcpyAsync(s_val_in.p, S->values, (size_t)snz * vb,
                                     S->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    }
    SDA_CUDA(cudaMemcpyAsync(&ends[0], op->s_rp.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaMemcpyAsync(&ends[1], op->s_rp.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    if (ends[0] != 0 || ends[1] != snz)
        return fail(SDA_ERR_INDEX, "S row_ptr must start at 0 and end at nnz");
    k_check_csr<<<grid1(n, sms), kBlock, 0, s>>>(n, n, op->s_rp.p, op->s_col.p, S->values ? s_val_in.p : nullptr,
                                                 s_in_dt, 1, err.p);
    SDA_LAUNCHED();
    SDA_TRY(read_err(err, s, &herr));
    if (herr & (kErrIndex | kErrRowPtr)) return fail(SDA_ERR_INDEX, "S: bad row pointers or column indices");
    if (herr & (kErrWeight | kErrNonFinite)) return fail(SDA_ERR_NOT_SYMMETRIC, "S holds a negative or non-finite weight");
    {
        DevBuf<uint32_t> keys, vals;
        DevBuf<int32_t> row_of;
        SDA_TRY(keys.alloc((size_t)std::max<int64_t>(snz, 1)));
        SDA_TRY(vals.alloc((size_t)std::max<int64_t>(snz, 1)));
        SDA_TRY(row_of.alloc((size_t)std::max<int64_t>(snz, 1)));
        k_relabel<<<grid1(snz, sms), kBlock, 0, s>>>(snz, op->s_col.p, nullptr, op->s_col.p, keys.p, vals.p);
        SDA_LAUNCHED();
        SDA_TRY(radix_sort_pairs(keys.p, vals.p, snz, bits_for((unsigned long long)std::max<int64_t>(n - 1, 1)), s));
        k_expand_rows<<<grid1(n, sms), kBlock, 0, s>>>(n, op->s_rp.p, row_of.p);
        SDA_LAUNCHED();
        k_check_sym<<<grid1(snz, sms), kBlock, 0, s>>>(snz, keys.p, vals.p, row_of.p, op->s_col.p,
                                                       S->values ? s_val_in.p : nullptr, s_in_dt, err.p);
        SDA_LAUNCHED();
        SDA_TRY(read_err(err, s, &herr));
        if (herr & kErrAsym) return fail(SDA_ERR_NOT_SYMMETRIC, "S is not equal to its transpose");
    }
    SDA_TRY(op->s_val64.alloc((size_t)std::max<int64_t>(snz, 1)));
    SDA_TRY(op->deg64.alloc((size_t)std::max<int64_t>(n, 1)));
    if (fp64) {
        k_degrees<double><<<grid1(n, sms), kBlock, 0, s>>>(n, op->s_rp.p, S->values ? s_val_in.p : nullptr, s_in_dt,
                                                           op->s_val64.p, nullptr, op->deg64.p, nullptr);
    } else {
        SDA_TRY(op->s_val32.alloc((size_t)std::max<int64_t>(snz, 1)));
        SDA_TRY(op->deg32.alloc((size_t)std::max<int64_t>(n, 1)));
        k_degrees<float><<<grid1(n, sms), kBlock, 0, s>>>(n, op->s_rp.p, S->values ? s_val_in.p : nullptr, s_in_dt,
                                                          op->s_val64.p, op->s_val32.p, op->deg64.p, op->deg32.p);
    }
    SDA_LAUNCHED();


    // ---- labels ----------------------------------------------------------------
    const int64_t T = y->n_targets;
    SDA_TRY(to_device(op->labels, y->labels, T * n, y->on_device, s));
    k_check_labels<<<grid1(T * n, sms), kBlock, 0, s>>>(T * n, op->labels.p, err.p);
    SDA_LAUNCHED();
    SDA_TRY(read_err(err, s, &herr));
    if (herr & kErrLabel) return fail(SDA_ERR_INVALID_ARG, "labels must be -1, 0 or +1");

    // ---- tile schedules of the sparse passes -------------------------------------
    {
        std::vector<int64_t> hp((size_t)std::max(n, d) + 1);
        hp.resize((size_t)d + 1);
        SDA_CUDA(cudaMemcpyAsync(hp.data(), op->x_cp.p, ((size_t)d + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        SDA_CUDA(cudaStreamSynchronize(s));
        SDA_TRY(build_seg_schedule(hp, op->col));
        // the columns after the head, for the batched column pass (segments from 0 = column hb.nseg)
        {
            std::vector<int64_t> tail(hp.begin() + op->hb.nseg, hp.end());
            SDA_TRY(build_seg_schedule(tail, op->col_tail));
        }
        hp.resize((size_t)n + 1);
        SDA_CUDA(cudaMemcpyAsync(hp.data(), op->x_rp.p, ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        SDA_CUDA(cudaStreamSynchronize(s));
        SDA_TRY(build_seg_schedule(hp, op->xrow));
        op->x_lanes = row_lanes(hp);
        SDA_CUDA(cudaMemcpyAsync(hp.data(), op->s_rp.p, ((size_t)n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        SDA_CUDA(cudaStreamSynchronize(s));
        SDA_TRY(build_seg_schedule(hp, op->srow));
        op->s_lanes = row_lanes(hp);
    }
    // split segments of the four schedules use disjoint slot / counter ranges
    op->xrow_slot0 = op->col.nslots;
    op->srow_slot0 = op->col.nslots + op->xrow.nslots;
    op->xb.slot0 = op->srow_slot0 + op->srow.nslots;
    op->xrow_lseg0 = op->col.nsplits;
    op->srow_lseg0 = op->col.nsplits + op->xrow.nsplits;
    op->xb.lseg0 = op->srow_lseg0 + op->srow.nsplits;
    SDA_TRY(op->slots.alloc((size_t)std::max(op->xb.slot0 + op->xb.sched.nslots, 1)));
    SDA_TRY(op->lcount.alloc((size_t)std::max(op->xb.lseg0 + op->xb.sched.nsplits, 1)));
    SDA_CUDA(cudaMemsetAsync(op->lcount.p, 0, op->lcount.bytes(), s));
    SDA_TRY(op->part.alloc((size_t)kMaxBlocksPerSm * op->sm_count * 4));
    SDA_TRY(op->cnt.alloc(4));
    SDA_CUDA(cudaMemsetAsync(op->cnt.p, 0, op->cnt.bytes(), s));
    SDA_TRY(op->scal.alloc(8));

    // ---- per-target counts and means (Alg. 7 step 3) ---------------------------------
    SDA_TRY(op->mu.alloc((size_t)(T * d)));
    SDA_TRY(op->mu32.alloc((size_t)(T * d)));
    SDA_TRY(op->dvec.alloc((size_t)(T * d)));
    op->counts.assign((size_t)T * 3, 0.0);
    if (op->regression) {
        // X^T X of the regression phase: every row counts, nothing is centred
        SDA_CUDA(cudaMemsetAsync(op->mu.p, 0, op->mu.bytes(), s));
        SDA_CUDA(cudaMemsetAsync(op->mu32.p, 0, op->mu32.bytes(), s));
        SDA_CUDA(cudaMemsetAsync(op->dvec.p, 0, op->dvec.bytes(), s));
        op->counts[0] = op->counts[1] = (double)n;
        SDA_CUDA(cudaStreamSynchronize(s));
        return SDA_OK;
    }
    {
        // class sums X^T 1_+ and X^T 1_- of up to eight targets per FP64 block
        // column pass (a single target: one plain column pass each)
        const int tg = T > 1 ? 8 : 1;
        DevBuf<double> ind, sums;
        DevBuf<unsigned long long> c2;
        SDA_TRY(ind.alloc((size_t)(2 * tg * n)));
        SDA_TRY(sums.alloc((size_t)(2 * tg * d)));
        SDA_TRY(c2.alloc((size_t)(2 * tg)));
        for (int64_t t0 = 0; t0 < T; t0 += tg) {
            const int nt = (int)std::min<int64_t>(tg, T - t0);
            const double *src[16];
            double *dst[16];
            SDA_CUDA(cudaMemsetAsync(c2.p, 0, (size_t)(2 * tg) * sizeof(unsigned long long), s));
            for (int k = 0; k < nt; ++k) {
                double *ip = ind.p + (int64_t)(2 * k) * n, *in_ = ip + n;
                k_indicators<<<grid1(n, sms), kBlock, 0, s>>>(n, op->labels.p + (t0 + k) * n, ip, in_, c2.p + 2 * k);
                SDA_LAUNCHED();
                src[2 * k] = ip;
                src[2 * k + 1] = in_;
                dst[2 * k] = sums.p + (int64_t)(2 * k) * d;
                dst[2 * k + 1] = dst[2 * k] + d;
            }
            if (T > 1) {
                SDA_TRY(xt_lanes(op, src, 2 * nt, dst, s));
            } else {
                SDA_TRY(op_xtmul_f64(op, src[0], dst[0], s));
                SDA_TRY(op_xtmul_f64(op, src[1], dst[1], s));
            }
            unsigned long long hc[16];
            SDA_CUDA(cudaMemcpyAsync(hc, c2.p, (size_t)(2 * nt) * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            SDA_CUDA(cudaStreamSynchronize(s));
            for (int k = 0; k < nt; ++k) {
                const int64_t t = t0 + k;
                if (hc[2 * k] == 0)
                    return fail(SDA_ERR_NO_POSITIVE, "target %lld has no labelled positive sample", (long long)t);
                if (hc[2 * k + 1] == 0)
                    return fail(SDA_ERR_NO_NEGATIVE, "target %lld has no labelled negative sample", (long long)t);
                op->counts[t * 3 + 0] = (double)(hc[2 * k] + hc[2 * k + 1]);
                op->counts[t * 3 + 1] = (double)hc[2 * k];
                op->counts[t * 3 + 2] = (double)hc[2 * k + 1];
                k_means<<<grid1(d, sms), kBlock, 0, s>>>(d, dst[2 * k], dst[2 * k + 1], (double)hc[2 * k],
                                                         (double)hc[2 * k + 1], op->mu.p + t * d, op->mu32.p + t * d,
                                                         op->dvec.p + t * d);
                SDA_LAUNCHED();
            }
        }
        SDA_CUDA(cudaStreamSynchronize(s));
    }
    return SDA_OK;
}

}  // namespace sda

using namespace sda;

static int build_entry(const sda_csr *X, const sda_csr *S, const sda_labels *y, double alpha,
                       double scatter_weight, sda_dtype compute, void *cuda_stream, sda_operator **out,
                       bool regression) {
    if (!out) return fail(SDA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!X || !S || !y) return fail(SDA_ERR_INVALID_ARG, "X, S and y must not be NULL");
    if (!X->row_ptr || (X->nnz > 0 && !X->col_idx) || !S->row_ptr || (S->nnz > 0 && !S->col_idx) || !y->labels)
        return fail(SDA_ERR_INVALID_ARG, "missing array");
    if (X->n_rows <= 0 || X->n_cols <= 0 || X->nnz < 0 || S->nnz < 0 || y->n_targets <= 0)
        return fail(SDA_ERR_SHAPE, "empty X or no targets");
    if (S->n_rows != X->n_rows || S->n_cols != X->n_rows)
        return fail(SDA_ERR_SHAPE, "S must be N x N with N = rows of X");
    if (X->n_cols > INT32_MAX || X->n_rows > INT32_MAX || X->nnz > (int64_t)UINT32_MAX || S->nnz > (int64_t)UINT32_MAX)
        return fail(SDA_ERR_SHAPE, "sizes beyond 32-bit indexing");
    if (X->values && X->dtype != SDA_F64 && X->dtype != SDA_F32)
        return fail(SDA_ERR_INVALID_ARG, "X values must be F64 or F32 (or NULL for a pattern)");
    if (S->values && S->dtype != SDA_F64 && S->dtype != SDA_F32)
        return fail(SDA_ERR_INVALID_ARG, "S values must be F64 or F32 (or NULL for all-ones weights)");
    if (compute < SDA_F64 || compute > SDA_PATTERN) return fail(SDA_ERR_INVALID_ARG, "bad compute dtype");
    if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(SDA_ERR_INVALID_ARG, "alpha must be in [0, 1]");
    const double omega = isnan(scatter_weight) ? 1.0 - alpha : scatter_weight;
    if (!(omega >= 0.0) || !isfinite(omega)) return fail(SDA_ERR_INVALID_ARG, "scatter weight must be >= 0");
    sda_operator *op = new (std::nothrow) sda_operator();
    if (!op) return fail(SDA_ERR_OOM, "host allocation failed");
    cudaGetDevice(&op->device);
    op->n = X->n_rows;
    op->d = X->n_cols;
    op->nnz = X->nnz;
    op->s_nnz = S->nnz;
    op->n_targets = y->n_targets;
    op->compute = compute;
    op->alpha = alpha;
    op->omega = omega;
    op->omega_follows_alpha = isnan(scatter_weight);
    op->regression = regression;
    op->sm_count = device_sm_count();
    if (op->sm_count <= 0) {
        delete op;
        return fail(SDA_ERR_CUDA, "no CUDA device");
    }
    op->grid = op->sm_count * 4;
    int rc = build(X, S, y, alpha, omega, compute, (cudaStream_t)cuda_stream, op);
    if (rc < 0) {
        cudaStreamSynchronize((cudaStream_t)cuda_stream);
        delete op;
        return rc;
    }
    op->bytes = (int64_t)(op->new_of_old.bytes() + op->old_of_new.bytes() + op->x_rp.bytes() + op->x_cp.bytes() +
                          op->x_col.bytes() + op->x_row.bytes() + op->x_val_r.bytes() + op->x_val_c.bytes() +
                          op->xb.bytes() + op->hb.cp.bytes() + op->hb.idx.bytes() + op->hb.val.bytes() +
                          op->xr_rp.bytes() + op->xr_col.bytes() + op->xr_val.bytes() +
                          op->s_rp.bytes() + op->s_col.bytes() + op->s_val64.bytes() + op->s_val32.bytes() +
                          op->deg64.bytes() + op->deg32.bytes() + op->labels.bytes() + op->mu.bytes() +
                          op->mu32.bytes() + op->dvec.bytes() + op->col.tiles.bytes() + op->col.splits.bytes() +
                          op->xrow.tiles.bytes() + op->xrow.splits.bytes() + op->srow.tiles.bytes() +
                          op->srow.splits.bytes());
    *out = op;
    return SDA_OK;
}

extern "C" SDA_API int sda_build_operator(const sda_csr *X, const sda_csr *S, const sda_labels *y, double alpha,
                                          double scatter_weight, sda_dtype compute, void *cuda_stream,
                                          sda_operator **out) {
    clear_error();
    return build_entry(X, S, y, alpha, scatter_weight, compute, cuda_stream, out, false);
}

extern "C" SDA_API int sda_build_regression(const sda_csr *X, sda_dtype compute, void *cuda_stream,
                                            sda_operator **out) {
    clear_error();
    if (!out) return fail(SDA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!X) return fail(SDA_ERR_INVALID_ARG, "X must not be NULL");
    if (X->n_rows <= 0 || X->n_rows > INT32_MAX) return fail(SDA_ERR_SHAPE, "X must have 1 .. 2^31 - 1 rows");
    // the SDA operator with an empty graph, every row labelled (P_l = I),
    // alpha = 0, omega = 1; the build then drops the centring (mu = 0)
    std::vector<int64_t> sp((size_t)X->n_rows + 1, 0);
    std::vector<int8_t> lab((size_t)X->n_rows, 1);
    const sda_csr S{X->n_rows, X->n_rows, 0, sp.data(), nullptr, nullptr, SDA_F64, 0};
    const sda_labels y{1, lab.data(), 0};
    return build_entry(X, &S, &y, 0.0, 1.0, compute, cuda_stream, out, true);
}

extern "C" SDA_API int sda_build_sa(const sda_csr *S, const sda_labels *y, double alpha, double scatter_weight,
                                    sda_dtype compute, void *cuda_stream, sda_operator **out) {
    clear_error();
    if (!out) return fail(SDA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!S) return fail(SDA_ERR_INVALID_ARG, "S must not be NULL");
    if (S->n_rows <= 0 || S->n_rows > INT32_MAX) return fail(SDA_ERR_SHAPE, "S must have 1 .. 2^31 - 1 rows");
    // the SDA operator with the identity as the data matrix (Algorithm 6): X = I_N
    const int64_t n = S->n_rows;
    std::vector<int64_t> xp((size_t)n + 1);
    std::vector<int32_t> xc((size_t)n);
    for (int64_t i = 0; i <= n; ++i) xp[(size_t)i] = i;
    for (int64_t i = 0; i < n; ++i) xc[(size_t)i] = (int32_t)i;
    const sda_csr X{n, n, n, xp.data(), xc.data(), nullptr, SDA_PATTERN, 0};
    return build_entry(&X, S, y, alpha, scatter_weight, compute, cuda_stream, out, false);
}
