// Shifted-CG solve driver (Algorithm 3 on the operator of Algorithm 7), the
// FP64 operator apply, projection, and the small ABI entry points.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "sda_kernels.cuh"

namespace sda {

int last_error(char *buf, int len);

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_dot_f64(int64_t n, const double *__restrict__ a,
                                                    const double *__restrict__ b, double *out,
                                                    double *partials, unsigned *counter) {
    __shared__ double red[kRedDoubles];
    double s[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock)
        s[0] += b ? a[i] * b[i] : a[i];
    double mine[1];
    block_dots<1>(s, mine, red);
    if (!arrive_last<1>(mine, partials, counter)) return;
    double tot[1];
    grid_dots<1>(partials, gridDim.x, tot, red);
    if (threadIdx.x == 0) {
        *out = tot[0];
        *counter = 0u;
    }
}

// ||b - q||^2 into *out
__global__ void __launch_bounds__(kBlock) k_resid_f64(int64_t n, const double *__restrict__ b,
                                                      const double *__restrict__ q, double *out,
                                                      double *partials, unsigned *counter) {
    __shared__ double red[kRedDoubles];
    double s[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) {
        const double e = b[i] - q[i];
        s[0] += e * e;
    }
    double mine[1];
    block_dots<1>(s, mine, red);
    if (!arrive_last<1>(mine, partials, counter)) return;
    double tot[1];
    grid_dots<1>(partials, gridDim.x, tot, red);
    if (threadIdx.x == 0) {
        *out = tot[0];
        *counter = 0u;
    }
}

__global__ void k_to_new(int64_t d, int64_t count, const int32_t *new_of_old, const double *in, double *out) {
    const int64_t m = d * count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / d, o = i - v * d;
        out[v * d + new_of_old[o]] = in[i];
    }
}

__global__ void k_to_old(int64_t d, int64_t count, const int32_t *new_of_old, const double *in, double *out) {
    const int64_t m = d * count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / d, o = i - v * d;
        out[i] = in[v * d + new_of_old[o]];
    }
}

// out[s][old] = W[s][new(old)] as FP64

template <class FT>
__global__ void k_w_f64(int64_t d, const FT *W, double *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)W[i];
}

// out = a x + b y
__global__ void k_axpby_f64(int64_t n, double a, const double *x, double b, const double *y, double *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a * x[i] + b * y[i];
}

// w += W (one shift's solution in the vector type)
template <class FT>
__global__ void k_add_w(int64_t d, const FT *W, double *w) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
        w[i] += (double)W[i];
}

__global__ void k_scale(int64_t d, const double *x, const double *coef, double mult, double *out) {
    const double c = *coef * mult;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = c * x[i];
}

// G[rows[h]] += g[h]; a row out of range sets *err
__global__ void k_scatter_rows(int64_t m, const int64_t *rows, const double *g, double *G, int64_t n, int *err) {
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < m; h += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = rows[h];
        if (i < 0 || i >= n) {
            atomicOr(err, 1);
            continue;
        }
        atomicAdd(G + i, g[h]);
    }
}

// c_j -= mu_j * (*t)
__global__ void k_sub_mu(int64_t d, double *c, const double *mu, const double *t) {
    const double tv = *t;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x)
        c[j] -= mu[j] * tv;
}

// out_i = [y_i != 0] u_i  (P_l u)
__global__ void k_mask_labelled(int64_t n, const int8_t *y, const double *u, double *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = y[i] != 0 ? u[i] : 0.0;
}

// WT[j][v] = w_v[old_of_new(j)]: nv vectors of the caller's feature order, transposed
// into the permuted order so that a row's entry reads its nv values contiguously
__global__ void k_to_new_t(int64_t d, int nv, const int32_t *new_of_old, const double *w, double *WT) {
    const int64_t m = d * nv;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / d, o = i - v * d;
        WT[(int64_t)new_of_old[o] * nv + v] = w[i];
    }
}

// part[b][v] = sum over the features j = b, b + nb, ... of mu_j WT[j][v] (fixed order)
__global__ void __launch_bounds__(kBlock) k_mu_dots_part(int64_t d, int nv, const double *__restrict__ mu,
                                                         const double *__restrict__ WT, double *__restrict__ part) {
    __shared__ double red[kBlock];
    for (int v0 = 0; v0 < nv; v0 += kBlock / 32) {
        const int v = v0 + (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
        double a = 0.0;
        if (v < nv)
            for (int64_t j = (int64_t)blockIdx.x * 32 + lane; j < d; j += (int64_t)gridDim.x * 32) a += mu[j] * WT[j * nv + v];
        a = warp_sum(a);
        if (lane == 0) red[threadIdx.x >> 5] = a;
        __syncthreads();
        if (threadIdx.x < kBlock / 32 && v0 + (int)threadIdx.x < nv)
            part[(int64_t)blockIdx.x * nv + v0 + threadIdx.x] = red[threadIdx.x];
        __syncthreads();
    }
}

// c[v] = sum_b part[b][v]
__global__ void k_mu_dots_sum(int nb, int nv, const double *__restrict__ part, double *__restrict__ c) {
    const int v = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (v >= nv) return;
    double a = 0.0;
    for (int b = 0; b < nb; ++b) a += part[(int64_t)b * nv + v];
    c[v] = a;
}

// scores[v][h] = sum over row rows[h] of x_e WT[col_e][v] (- c[v] when c is given):
// one warp per held row, its lanes over the vectors; a row id outside [0, n) sets *err
template <class VT>
__global__ void k_project_rows(int64_t n, int64_t nrows, int nv, const int64_t *__restrict__ rows,
                               const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                               const VT *__restrict__ val, const double *__restrict__ WT,
                               const double *__restrict__ c, double *__restrict__ scores, int *err) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t h = warp; h < nrows; h += nwarps) {
        const int64_t i = rows[h];
        if (i < 0 || i >= n) {
            if (lane == 0) atomicOr(err, 1);
            continue;
        }
        for (int v0 = 0; v0 < nv; v0 += 32) {
            const int v = v0 + lane;
            double a = 0.0;
            if (v < nv)
                for (int64_t e = rp[i]; e < rp[i + 1]; ++e) a += (double)Val<VT>::get(val, e) * WT[(int64_t)col[e] * nv + v];
            if (v < nv) scores[(int64_t)v * nrows + h] = c ? a - c[v] : a;
        }
    }
}

static int grid_elems(int64_t m, int sms) {
    const int64_t g = (m + kBlock - 1) / kBlock;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)sms * 16));
}

// ---------------------------------------------------------------------------
// dispatch helpers
// ---------------------------------------------------------------------------
template <class F>
static int with_vt(int compute, F &&f) {
    switch (compute) {
    case SDA_F64: return f((double *)nullptr);
    case SDA_F32: return f((float *)nullptr);
    case SDA_F16: return f((__half *)nullptr);
    case SDA_F8E4M3: return f((__nv_fp8_e4m3 *)nullptr);
    case SDA_PATTERN: return f((Pattern *)nullptr);
    default: return fail(SDA_ERR_INVALID_ARG, "bad compute dtype");
    }
}

// lanes per row G and unrolled loads per lane U of the register row pass
template <class F>
static int with_row_lanes(int g, F &&f) {
    switch (g) {
    case 4: return f(std::integral_constant<int, 4>(), std::integral_constant<int, 4>());
    case 8: return f(std::integral_constant<int, 8>(), std::integral_constant<int, 4>());
    case 16: return f(std::integral_constant<int, 16>(), std::integral_constant<int, 4>());
    default: return f(std::integral_constant<int, 32>(), std::integral_constant<int, 4>());
    }
}

template <class F>
static int with_quad_lanes(int g, F &&f) {
    switch (g) {
    case 2: return f(std::integral_constant<int, 2>());
    case 4: return f(std::integral_constant<int, 4>());
    case 8: return f(std::integral_constant<int, 8>());
    case 16: return f(std::integral_constant<int, 16>());
    default: return f(std::integral_constant<int, 32>());
    }
}

// ---------------------------------------------------------------------------
// FP64 operator pieces (permuted feature order)
// ---------------------------------------------------------------------------
// a sparse pass with one of the operator's schedules
template <class VT, class AccT, class Gather, class Epi>
static int segpass(const sda_operator *op, const ColSchedule &sc, int32_t slot0, int32_t lseg0,
                   const int64_t *ptr, const int32_t *idx, const void *val, const Gather &g, const Epi &e,
                   int grid, cudaStream_t s) {
    k_segpass<VT, AccT, Gather, Epi><<<grid, kBlock, 0, s>>>(sc.tiles.p, sc.ntiles, ptr, idx, (const VT *)val, g, e,
                                                            (AccT *)op->slots.p + slot0, op->lcount.p + lseg0,
                                                            sc.splits.p);
    SDA_LAUNCHED();
    return SDA_OK;
}

// a column pass over X^T with the operator's column schedule
template <class VT, class AccT, class Epi>
static int colpass(const sda_operator *op, const AccT *v, const Epi &e, int grid, cudaStream_t s) {
    k_colpass<VT, AccT, 8, Epi><<<grid, kBlock, 0, s>>>(op->col.tiles.p, op->col.ntiles, op->x_cp.p, op->x_row.p,
                                                       (const VT *)op->x_val_c.p, v, (AccT *)op->slots.p,
                                                       op->lcount.p, op->col.splits.p, e);
    SDA_LAUNCHED();
    return SDA_OK;
}

int op_xtmul_f64(const sda_operator *op, const double *v, double *q, cudaStream_t s) {
    return with_vt(op->compute, [&](auto tag) -> int {
        using VT = std::remove_pointer_t<decltype(tag)>;
        return colpass<VT, double>(op, v, EpiStore<double>{q, nullptr, nullptr, 0.0}, op->sm_count * kMaxBlocksPerSm,
                                   s);
    });
}

// a register row pass over the rows of a CSR matrix
template <class VT, class AccT, class Gather, class Epi>
static int rowpass(int lanes, int64_t n, const int64_t *rp, const int32_t *idx, const void *val, const Gather &g,
                   const Epi &e, int grid, cudaStream_t s) {
    return with_row_lanes(lanes, [&](auto G, auto U) -> int {
        k_rowpass<VT, AccT, decltype(G)::value, decltype(U)::value, Gather, Epi>
            <<<grid, kBlock, 0, s>>>(n, rp, idx, (const VT *)val, g, e);
        SDA_LAUNCHED();
        return SDA_OK;
    });
}

int op_xmul_f64(const sda_operator *op, const double *w, double *u, const double *csub, cudaStream_t s) {
    return with_vt(op->compute, [&](auto tag) -> int {
        using VT = std::remove_pointer_t<decltype(tag)>;
        return rowpass<VT, double>(op->x_lanes, op->n, op->x_rp.p, op->x_col.p, op->x_val_r.p,
                                   GatherVec<double, double>{w}, EpiStore<double>{u, csub, nullptr, 0.0},
                                   op->sm_count * kMaxBlocksPerSm, s);
    });
}

int dot_f64(const sda_operator *op, int64_t n, const double *a, const double *b, double *out, cudaStream_t s) {
    k_dot_f64<<<op->grid, kBlock, 0, s>>>(n, a, b, out, op->part.p, op->cnt.p);
    SDA_LAUNCHED();
    return SDA_OK;
}

static int ensure_apply_scratch(sda_operator *op) {
    Workspace &w = op->ws;
    const size_t need = (size_t)(3 * op->d + 2 * op->n);
    if (w.f64.n < need) SDA_TRY(w.f64.alloc(need));
    return SDA_OK;
}

// q = (B + sigma I) p, FP64, centred symmetric form, permuted order, at (alpha, omega)
int op_apply_f64(const sda_operator *op, int target, double sigma, const double *p, double *q, cudaStream_t s,
                 double alpha, double omega) {
    sda_operator *mop = const_cast<sda_operator *>(op);
    SDA_TRY(ensure_apply_scratch(mop));
    double *u = op->ws.f64.p + 3 * op->d, *v = u + op->n;
    const double *mu = op->mu.p + (int64_t)target * op->d;
    const int8_t *y = op->labels.p + (int64_t)target * op->n;
    SDA_TRY(dot_f64(op, op->d, mu, p, op->scal.p + 0, s));
    SDA_TRY(op_xmul_f64(op, p, u, op->scal.p + 0, s));
    SDA_TRY((rowpass<double, double>(op->s_lanes, op->n, op->s_rp.p, op->s_col.p, op->s_val64.p,
                                     GatherVec<double, double>{u}, EpiLap64{v, u, op->deg64.p, y, omega, alpha},
                                     op->sm_count * kMaxBlocksPerSm, s)));
    SDA_TRY(dot_f64(op, op->n, v, nullptr, op->scal.p + 1, s));
    return with_vt(op->compute, [&](auto tag) -> int {
        using VT = std::remove_pointer_t<decltype(tag)>;
        return colpass<VT, double>(op, v, EpiApply{q, mu, p, op->scal.p + 1, sigma, 0.0},
                                   op->sm_count * kMaxBlocksPerSm, s);
    });
}

int permute_to_new(const sda_operator *op, const double *in, double *out, int64_t count, cudaStream_t s) {
    k_to_new<<<grid_elems(op->d * count, op->sm_count), kBlock, 0, s>>>(op->d, count, op->new_of_old.p, in, out);
    SDA_LAUNCHED();
    return SDA_OK;
}

int permute_to_old(const sda_operator *op, const double *in, double *out, int64_t count, cudaStream_t s) {
    k_to_old<<<grid_elems(op->d * count, op->sm_count), kBlock, 0, s>>>(op->d, count, op->new_of_old.p, in, out);
    SDA_LAUNCHED();
    return SDA_OK;
}

// ---------------------------------------------------------------------------
// solve workspace
// ---------------------------------------------------------------------------
void release_workspace(sda_operator *op) {
    Workspace &w = op->ws;
    if (w.graph) cudaGraphExecDestroy(w.graph);
    w.graph = nullptr;
    w.graph_iters = 0;
    if (w.cap_stream) cudaStreamDestroy(w.cap_stream);
    w.cap_stream = nullptr;
    if (w.h_st) cudaFreeHost(w.h_st);
    w.h_st = nullptr;
    for (cudaEvent_t e : w.prof_ev) cudaEventDestroy(e);
    w.prof_ev.clear();
    for (cudaEvent_t &e : w.call_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    w.vec.release();
    w.shift.release();
    w.st.release();
    w.part.release();
    w.cnt.release();
    w.f64.release();
    w.w64.release();
    w.dev_b.release();
}

static int ensure_workspace(sda_operator *op, int ns) {
    Workspace &w = op->ws;
    const int fp64 = op->compute == SDA_F64;
    const size_t fsz = fp64 ? sizeof(double) : sizeof(float);
    const int64_t ldw = (op->d + 7) / 8 * 8;
    const int64_t n8 = (op->n + 7) / 8 * 8;
    const bool realloc = w.fp64 != fp64 || w.d != op->d || w.n != op->n || w.n_shifts < ns ||
                         w.nparts != op->xb.nranges;
    if (!realloc) return SDA_OK;
    if (w.graph) cudaGraphExecDestroy(w.graph);
    w.graph = nullptr;
    w.graph_iters = 0;
    // range partials are CompSum parts: two vector-type words each
    SDA_TRY(w.vec.alloc((size_t)((4 + 2 * op->xb.nranges) * ldw + 2 * n8) * fsz));
    SDA_TRY(w.shift.alloc((size_t)(2 * (int64_t)ns * ldw) * fsz));
    SDA_TRY(w.st.alloc(1));
    SDA_TRY(w.part.alloc((size_t)3 * kMaxBlocksPerSm * op->sm_count * 4));
    SDA_TRY(w.cnt.alloc(4));
    SDA_CUDA(cudaMemset(w.cnt.p, 0, w.cnt.bytes()));
    SDA_TRY(ensure_apply_scratch(op));
    if (!w.h_st) SDA_CUDA(cudaMallocHost(&w.h_st, sizeof(SolveState)));
    w.fp64 = fp64;
    w.d = op->d;
    w.n = op->n;
    w.ldw = ldw;
    w.n_shifts = ns;
    w.nparts = op->xb.nranges;
    w.vt = -1;
    return SDA_OK;
}

template <class FT>
struct WsView {
    typename RPair<FT>::T *rp;
    typename CompSum<FT>::Part *s;     // [nparts][ldw] range partials of X^T v
    FT *ut, *v, *W, *P;
};

template <class FT>
static WsView<FT> view(const sda_operator *op) {
    const Workspace &w = op->ws;
    FT *base = (FT *)w.vec.p;
    FT *sb = (FT *)w.shift.p;
    const int64_t l = w.ldw, n8 = (op->n + 7) / 8 * 8;
    using Part = typename CompSum<FT>::Part;
    FT *ut = base + (4 + 2 * w.nparts) * l;
    return WsView<FT>{(typename RPair<FT>::T *)base, (Part *)(base + 4 * l), ut, ut + n8, sb,
                      sb + (int64_t)w.n_shifts * l};
}

static int grid_of(const void *kernel, int sms) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kBlock, 0) != cudaSuccess || nb <= 0) {
        (void)cudaGetLastError();
        nb = 1;
    }
    return std::min(nb, kMaxBlocksPerSm) * sms;
}

// out[r * ldo + j] = sum over the entries of segment j in range r of value * v[row]
template <class VT, class FT>
static int range_pass(const sda_operator *op, const RangeBlocks &rb, int64_t n, int64_t nseg, int64_t ldo,
                      const FT *v, typename CompSum<FT>::Part *out, int grid, size_t smem, cudaStream_t s,
                      const typename RPair<FT>::T *rp, FT *W, FT *P, const void *p2parts, int p2blocks) {
    using Part = typename CompSum<FT>::Part;   // one slot (8 bytes) per part in either type
    k_colblk<VT, FT><<<grid, kColBlk, smem, s>>>(rb.sched.tiles.p, rb.per_range, n, rb.rb, nseg, ldo, rb.cp.p,
                                                 rb.idx.p, (const VT *)rb.val.p, v, out,
                                                 reinterpret_cast<Part *>(op->slots.p) + rb.slot0,
                                                 op->lcount.p + rb.lseg0, rb.sched.splits.p, rb.tile_off.p,
                                                 op->ws.st.p, ldo, rp, W, P,
                                                 (const typename CompSum<FT>::Part *)p2parts, p2blocks);
    SDA_LAUNCHED();
    return SDA_OK;
}

// value type of the blocked column layout (a pattern X stores FP8 ones there)
template <class VT>
using BlkVT = std::conditional_t<std::is_same<VT, Pattern>::value, __nv_fp8_e4m3, VT>;

// sizes the grids of the iteration kernels for this operator's dtypes
template <class VT, class FT>
static int size_grids(sda_operator *op) {
    Workspace &w = op->ws;
    if (w.vt == (int)op->compute) return SDA_OK;
    const int sms = op->sm_count;
    SDA_TRY(with_quad_lanes(op->xr_lanes, [&](auto G) -> int {
        const void *k = (const void *)k_rowhead<BlkVT<VT>, FT, decltype(G)::value>;
        const size_t smem = (size_t)op->xr_head * sizeof(FT);
        SDA_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int nb = 0;
        SDA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kColBlk, smem));
        if (nb <= 0) return fail(SDA_ERR_UNSUPPORTED, "the row pass does not fit on an SM");
        w.grid1 = nb * sms;
        w.rowhead_smem = smem;
        return SDA_OK;
    }));
    SDA_TRY(with_row_lanes(op->s_lanes, [&](auto G, auto U) -> int {
        w.grid2 = grid_of((const void *)k_rowpass<FT, FT, decltype(G)::value, decltype(U)::value, GatherVec<FT, FT>,
                                                  EpiP2<FT>>, sms);
        return SDA_OK;
    }));
    {
        const void *k = (const void *)k_colblk<BlkVT<VT>, FT>;
        const size_t smem = ((size_t)op->xb.rb * sizeof(FT) + 15) / 16 * 16 + (size_t)colblk_scratch(sizeof(FT));
        SDA_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int nb = 0;
        SDA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kColBlk, smem));
        if (nb <= 0) return fail(SDA_ERR_UNSUPPORTED, "the column pass does not fit on an SM");
        w.colblk_smem = smem;
        w.grid3a = op->xb.per_range * op->xb.nranges;
    }
    w.grid3b = grid_of((const void *)k_cg_phase3b<FT>, sms);
    w.vt = (int)op->compute;
    return SDA_OK;
}

// the four kernels of one iteration; `ev` (profile mode) holds a start and an
// end event for each of them
template <class VT, class FT>
static int launch_iteration(const sda_operator *op, cudaStream_t s, cudaEvent_t *ev = nullptr) {
    const Workspace &w = op->ws;
    WsView<FT> b = view<FT>(op);
    const FT *dg = std::is_same<FT, double>::value ? (const FT *)op->deg64.p : (const FT *)op->deg32.p;
    const size_t P = (size_t)kMaxBlocksPerSm * op->sm_count;
    if (ev) SDA_CUDA(cudaEventRecord(ev[0], s));
    SDA_TRY(with_quad_lanes(op->xr_lanes, [&](auto G) -> int {
        k_rowhead<BlkVT<VT>, FT, decltype(G)::value><<<w.grid1, kColBlk, w.rowhead_smem, s>>>(
            op->n, op->xr_head, w.ldw, op->xr_rp.p, op->xr_col.p, (const BlkVT<VT> *)op->xr_val.p, b.rp, b.ut,
            w.st.p);
        SDA_LAUNCHED();
        return SDA_OK;
    }));
    if (ev) SDA_CUDA(cudaEventRecord(ev[1], s));
    if (ev) SDA_CUDA(cudaEventRecord(ev[2], s));
    const FT *sv = std::is_same<FT, double>::value ? (const FT *)op->s_val64.p : (const FT *)op->s_val32.p;
    SDA_TRY((rowpass<FT, FT>(op->s_lanes, op->n, op->s_rp.p, op->s_col.p, sv, GatherVec<FT, FT>{b.ut},
                             EpiP2<FT>{b.v, b.ut, dg, w.st.p, w.part.p + P * 4, nullptr, 0, 0},
                             w.grid2, s)));
    if (ev) SDA_CUDA(cudaEventRecord(ev[3], s));
    if (ev) SDA_CUDA(cudaEventRecord(ev[4], s));
    SDA_TRY((range_pass<BlkVT<VT>, FT>(op, op->xb, op->n, op->d, w.ldw, b.v, b.s, w.grid3a, w.colblk_smem, s, b.rp,
                                       b.W, b.P, w.part.p + P * 4, w.grid2)));
    if (ev) SDA_CUDA(cudaEventRecord(ev[5], s));
    if (ev) SDA_CUDA(cudaEventRecord(ev[6], s));
    k_cg_phase3b<FT><<<w.grid3b, kBlock, 0, s>>>(op->d, w.ldw, b.s, w.nparts, b.rp, b.W, b.P, w.st.p,
                                                 w.part.p + P * 8, w.cnt.p + 2);
    SDA_LAUNCHED();
    if (ev) SDA_CUDA(cudaEventRecord(ev[7], s));
    return SDA_OK;
}

template <class VT, class FT>
static int run_iterations(sda_operator *op, int nb, bool use_graph, bool profile, cudaStream_t s) {
    Workspace &w = op->ws;
    if (profile) {
        const size_t need = (size_t)nb * 8;
        while (w.prof_ev.size() < need) {
            cudaEvent_t e;
            SDA_CUDA(cudaEventCreate(&e));
            w.prof_ev.push_back(e);
        }
        for (int i = 0; i < nb; ++i) SDA_TRY((launch_iteration<VT, FT>(op, s, w.prof_ev.data() + 8 * i)));
        SDA_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < nb; ++i)
            for (int ph = 0; ph < 4; ++ph) {
                float ms = 0.f;
                SDA_CUDA(cudaEventElapsedTime(&ms, w.prof_ev[8 * i + 2 * ph], w.prof_ev[8 * i + 2 * ph + 1]));
                op->stats.ms[1 + ph] += ms;
            }
        for (int ph = 1; ph <= 4; ++ph) op->stats.launches[ph] += nb;
        return SDA_OK;
    }
    if (!use_graph) {
        for (int i = 0; i < nb; ++i) SDA_TRY((launch_iteration<VT, FT>(op, s)));
        for (int ph = 1; ph <= 4; ++ph) op->stats.launches[ph] += nb;
        return SDA_OK;
    }
    if (!w.graph || w.graph_iters != nb) {
        if (w.graph) cudaGraphExecDestroy(w.graph);
        w.graph = nullptr;
        if (!w.cap_stream) SDA_CUDA(cudaStreamCreateWithFlags(&w.cap_stream, cudaStreamNonBlocking));
        SDA_CUDA(cudaStreamBeginCapture(w.cap_stream, cudaStreamCaptureModeThreadLocal));
        set_capturing(true);
        int rc = SDA_OK;
        for (int i = 0; i < nb && rc == SDA_OK; ++i) rc = launch_iteration<VT, FT>(op, w.cap_stream);
        set_capturing(false);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(w.cap_stream, &g);
        if (rc != SDA_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        e = cudaGraphInstantiate(&w.graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
        w.graph_iters = nb;
    }
    SDA_CUDA(cudaGraphLaunch(w.graph, s));
    note_launch(4 * (int64_t)nb);
    for (int ph = 1; ph <= 4; ++ph) op->stats.launches[ph] += nb;
    return SDA_OK;
}

static int read_header(sda_operator *op, cudaStream_t s) {
    Workspace &w = op->ws;
    const size_t hdr = offsetof(SolveState, sh);
    SDA_CUDA(cudaMemcpyAsync(w.h_st, w.st.p, hdr, cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    return SDA_OK;
}

// One shifted-CG run (Algorithm 3) on (B + beta I) w = b for the given shifts;
// the solutions stay in the workspace's W in the vector type, the final header
// and shift states in w.h_st.
template <class VT, class FT>
static int run_shifted(sda_operator *op, int t, const double *b_perm, const double *shifts, int ns, double tol,
                       int limit, bool fixed, const sda_solve_opts &o, double alpha, double omega, cudaStream_t s,
                       int *worst) {
    Workspace &w = op->ws;
    SDA_TRY((size_grids<VT, FT>(op)));
    WsView<FT> bv = view<FT>(op);
    SolveState &h = *w.h_st;
    memset(&h, 0, sizeof(SolveState));
    double sigma0 = shifts[0];
    for (int i = 1; i < ns; ++i) sigma0 = std::min(sigma0, shifts[i]);
    h.sigma0 = sigma0;
    h.omega = omega;
    h.alpha_l = alpha;
    h.tol = tol;
    h.n_shifts = ns;
    h.fixed = fixed ? 1 : 0;
    h.limit = limit;
    h.labels = op->labels.p + (int64_t)t * op->n;
    h.mu = op->mu.p + (int64_t)t * op->d;
    h.mu32 = op->mu32.p + (int64_t)t * op->d;
    for (int i = 0; i < ns; ++i) h.sh[i].delta = shifts[i] - sigma0;
    SDA_CUDA(cudaMemcpyAsync(w.st.p, &h, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    k_cg_init<FT><<<w.grid3b, kBlock, 0, s>>>(op->d, w.ldw, b_perm, bv.rp, bv.W, bv.P, w.st.p, w.part.p,
                                              w.cnt.p + 0);
    SDA_LAUNCHED();
    op->stats.launches[0] += 1;
    SDA_TRY(read_header(op, s));
    // iterations in batches; kernels of a finished run return at once, so a
    // batch may overshoot the stop by a few empty launches
    const int nb = o.iter_batch > 0 ? o.iter_batch : 32;
    int launched = 0;
    while (!h.done && launched <= h.limit) {
        SDA_TRY((run_iterations<VT, FT>(op, nb, o.use_graph != 0, o.profile != 0, s)));
        launched += nb;
        SDA_TRY(read_header(op, s));
    }
    if (h.status != SDA_OK) {
        *worst = h.status;
        fail(h.status, "breakdown in the shifted CG of target %d at iteration %d", t, h.k);
    }
    SDA_CUDA(cudaMemcpyAsync(w.h_st, w.st.p, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    op->stats.iterations += h.k;
    for (int i = 0; i < ns; ++i) op->stats.shift_iterations += h.sh[i].iters;
    return SDA_OK;
}

// ||b - (B + beta I) w|| squared into *out (FP64, permuted order)
int resid2(sda_operator *op, int t, double beta, const double *b_perm, const double *w64, double *out,
           double alpha, double omega, cudaStream_t s) {
    double *q = op->ws.f64.p + op->d;
    SDA_TRY(op_apply_f64(op, t, beta, w64, q, s, alpha, omega));
    k_resid_f64<<<op->grid, kBlock, 0, s>>>(op->d, b_perm, q, out, op->part.p, op->cnt.p);
    SDA_LAUNCHED();
    return SDA_OK;
}

template <class VT, class FT>
static int solve_target(sda_operator *op, int t, const double *b_perm, const double *shifts, int ns,
                        const sda_solve_opts &o, double alpha, double omega, double *w_out_t,
                        sda_shift_report *rep_t, cudaStream_t s, int *worst) {
    Workspace &w = op->ws;
    const int64_t d = op->d;
    const bool fixed = o.fixed_iters > 0;
    SDA_TRY((run_shifted<VT, FT>(op, t, b_perm, shifts, ns, o.tol, fixed ? o.fixed_iters : o.max_iter, fixed, o,
                                 alpha, omega, s, worst)));
    const SolveState outer = *w.h_st;
    const int rounds = fixed ? 0 : std::max(0, o.refine_rounds);
    const double rtol = std::isnan(o.refine_tol) || o.refine_tol <= 0.0 ? o.tol : o.refine_tol;
    const bool check = o.check_residual != 0 || rounds > 0;
    // the solutions in FP64 (refinement adds its corrections there)
    if (w.w64.n < (size_t)ns * (size_t)d + d) SDA_TRY(w.w64.alloc((size_t)ns * (size_t)d + d));
    double *W64 = w.w64.p, *rvec = w.w64.p + (int64_t)ns * d;
    {
        WsView<FT> bv = view<FT>(op);
        for (int i = 0; i < ns; ++i) {
            k_w_f64<FT><<<grid_elems(d, op->sm_count), kBlock, 0, s>>>(d, bv.W + (int64_t)i * w.ldw,
                                                                       W64 + (int64_t)i * d);
            SDA_LAUNCHED();
        }
    }
    // FP64 true residual of every shift, and per-shift refinement (mixed
    // precision: r = b - (B + beta) w in FP64, a single-shift solve of the
    // correction in the iteration's precision, w += correction in FP64)
    std::vector<double> tres((size_t)ns, -1.0);
    std::vector<int> rstatus((size_t)ns, SDA_OK);
    if (check) {
        DevBuf<double> rs;
        SDA_TRY(rs.alloc((size_t)ns + 1));
        SDA_TRY(dot_f64(op, d, b_perm, b_perm, rs.p + ns, s));
        SDA_TRY(resid_block(op, t, shifts, ns, b_perm, W64, rs.p, alpha, omega, s));
        std::vector<double> hr((size_t)ns + 1);
        SDA_CUDA(cudaMemcpyAsync(hr.data(), rs.p, hr.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        SDA_CUDA(cudaStreamSynchronize(s));
        const double bn = sqrt(hr[ns]);
        for (int i = 0; i < ns; ++i) tres[i] = bn > 0 ? sqrt(hr[i]) / bn : sqrt(hr[i]);
        for (int i = 0; i < ns; ++i) {
            for (int rd = 0; rd < rounds && tres[i] > rtol && bn > 0; ++rd) {
                double *wi = W64 + (int64_t)i * d;
                double *q = op->ws.f64.p + d;
                SDA_TRY(op_apply_f64(op, t, shifts[i], wi, q, s, alpha, omega));
                k_axpby_f64<<<grid_elems(d, op->sm_count), kBlock, 0, s>>>(d, 1.0, b_perm, -1.0, q, rvec);
                SDA_LAUNCHED();
                // relative reduction asked of the correction solve: to the target,
                // but not below what the iteration's precision can reach
                const double inner = std::min(0.5, std::max(rtol / tres[i], 1e-4));
                int iw = SDA_OK;
                SDA_TRY((run_shifted<VT, FT>(op, t, rvec, &shifts[i], 1, inner, o.max_iter, false, o, alpha, omega,
                                             s, &iw)));
                if (iw != SDA_OK) {
                    rstatus[i] = iw;
                    break;
                }
                WsView<FT> bv = view<FT>(op);
                k_add_w<FT><<<grid_elems(d, op->sm_count), kBlock, 0, s>>>(d, bv.W, wi);
                SDA_LAUNCHED();
                SDA_TRY(resid2(op, t, shifts[i], b_perm, wi, rs.p + i, alpha, omega, s));
                double r2 = 0.0;
                SDA_CUDA(cudaMemcpyAsync(&r2, rs.p + i, sizeof(double), cudaMemcpyDeviceToHost, s));
                SDA_CUDA(cudaStreamSynchronize(s));
                tres[i] = sqrt(r2) / bn;
            }
        }
        if (!o.check_residual && rounds == 0) std::fill(tres.begin(), tres.end(), -1.0);
    }
    // solution out, in the caller's feature order
    if (w_out_t) {
        double *dst = w_out_t;
        DevBuf<double> hostbuf;
        if (!o.out_on_device) {
            SDA_TRY(hostbuf.alloc((size_t)ns * d));
            dst = hostbuf.p;
        }
        SDA_TRY(permute_to_old(op, W64, dst, ns, s));
        if (!o.out_on_device) {
            SDA_CUDA(cudaMemcpyAsync(w_out_t, dst, (size_t)ns * d * sizeof(double), cudaMemcpyDeviceToHost, s));
            SDA_CUDA(cudaStreamSynchronize(s));
        }
    }
    for (int i = 0; i < ns; ++i) {
        const ShiftState &sh = outer.sh[i];
        int st = SDA_OK;
        if (outer.status != SDA_OK) st = outer.status;
        else if (rstatus[i] != SDA_OK) st = rstatus[i];
        else if (rounds > 0) st = tres[i] <= rtol ? SDA_OK : SDA_NOT_CONVERGED;
        else if (!fixed && sh.active) st = SDA_NOT_CONVERGED;
        if (st == SDA_NOT_CONVERGED && *worst == SDA_OK) *worst = SDA_NOT_CONVERGED;
        if (st < 0 && *worst >= 0) *worst = st;
        if (rep_t) {
            rep_t[i].iters = sh.iters;
            rep_t[i].status = st;
            rep_t[i].est_residual = sh.res;
            rep_t[i].true_residual = tres[i];
        }
    }
    return SDA_OK;
}

}  // namespace sda

using namespace sda;

extern "C" SDA_API void sda_default_opts(sda_solve_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->tol = 1e-6;
    o->max_iter = 10000;
    o->fixed_iters = 0;
    o->rhs_mode = SDA_RHS_CANONICAL;
    o->rhs = nullptr;
    o->target_begin = 0;
    o->target_count = -1;
    o->check_residual = 1;
    o->out_on_device = 1;
    o->use_graph = 1;
    o->iter_batch = 0;
    o->profile = 0;
    o->alpha = NAN;
    o->scatter_weight = NAN;
    o->refine_rounds = 0;
    o->batch_targets = 0;
    o->refine_tol = NAN;
    o->shift_form = SDA_SHIFTS_AUTO;
}

// the (alpha, omega) of a call: overrides from the options, else the operator's
static int call_weights(const sda_operator *op, const sda_solve_opts &o, double *alpha, double *omega) {
    const double a = isnan(o.alpha) ? op->alpha : o.alpha;
    if (!(a >= 0.0 && a <= 1.0)) return fail(SDA_ERR_INVALID_ARG, "alpha must be in [0, 1]");
    double w = o.scatter_weight;
    if (isnan(w)) w = op->omega_follows_alpha ? 1.0 - a : op->omega;
    if (!(w >= 0.0) || !isfinite(w)) return fail(SDA_ERR_INVALID_ARG, "scatter weight must be >= 0");
    *alpha = a;
    *omega = w;
    return SDA_OK;
}

extern "C" SDA_API int sda_solve_shifts(sda_operator *op, const double *shifts, int32_t n_shifts,
                                        const sda_solve_opts *opt, double *w_out, sda_shift_report *report,
                                        void *cuda_stream) {
    clear_error();
    if (!op || !shifts) return fail(SDA_ERR_INVALID_ARG, "operator and shifts must not be NULL");
    SDA_TRY(check_device(op->device));
    if (n_shifts < 1 || n_shifts > kMaxShifts) return fail(SDA_ERR_INVALID_ARG, "n_shifts must be in [1, %d]", kMaxShifts);
    for (int i = 0; i < n_shifts; ++i)
        if (!(shifts[i] > 0.0) || !isfinite(shifts[i])) return fail(SDA_ERR_INVALID_ARG, "shifts must be finite and > 0");
    sda_solve_opts o;
    if (opt) o = *opt;
    else sda_default_opts(&o);
    if (o.fixed_iters <= 0 && (!(o.tol >= 0.0) || o.max_iter < 0))
        return fail(SDA_ERR_INVALID_ARG, "tol must be >= 0 and max_iter >= 0");
    if (o.refine_rounds < 0) return fail(SDA_ERR_INVALID_ARG, "refine_rounds must be >= 0");
    if (o.shift_form < SDA_SHIFTS_AUTO || o.shift_form > SDA_SHIFTS_BASIS)
        return fail(SDA_ERR_INVALID_ARG, "bad shift_form");
    if (o.shift_form == SDA_SHIFTS_BASIS && !o.batch_targets)
        return fail(SDA_ERR_UNSUPPORTED, "the stored-basis shift form is provided on the batched path");
    const int t0 = o.target_begin;
    const int tc = o.target_count < 0 ? op->n_targets - t0 : o.target_count;
    if (t0 < 0 || tc < 0 || t0 + tc > op->n_targets) return fail(SDA_ERR_INVALID_ARG, "target range out of bounds");
    if (o.rhs_mode != SDA_RHS_CANONICAL && !o.rhs) return fail(SDA_ERR_INVALID_ARG, "rhs is NULL");
    if (o.rhs_mode < 0 || o.rhs_mode > SDA_RHS_GIVEN) return fail(SDA_ERR_INVALID_ARG, "bad rhs_mode");
    if (op->regression && (o.rhs_mode != SDA_RHS_GIVEN || !isnan(o.alpha) || !isnan(o.scatter_weight)))
        return fail(SDA_ERR_INVALID_ARG, "a regression operator takes a given right-hand side and no weights");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double alpha = 0.0, omega = 0.0;
    SDA_TRY(call_weights(op, o, &alpha, &omega));
    SDA_TRY(ensure_workspace(op, n_shifts));
    Workspace &w = op->ws;
    memset(&op->stats, 0, sizeof(op->stats));
    if (!w.call_ev[0]) {
        SDA_CUDA(cudaEventCreate(&w.call_ev[0]));
        SDA_CUDA(cudaEventCreate(&w.call_ev[1]));
    }
    SDA_CUDA(cudaEventRecord(w.call_ev[0], s));
    // right-hand sides in the permuted order
    const int64_t d = op->d;
    if (o.rhs_mode != SDA_RHS_CANONICAL) {
        SDA_TRY(w.dev_b.alloc((size_t)(o.rhs_mode == SDA_RHS_GIVEN ? tc : 1) * d));
        DevBuf<double> tmp;
        const double *src = o.rhs;
        const int64_t cnt = o.rhs_mode == SDA_RHS_GIVEN ? tc : 1;
        if (!o.rhs_on_device) {
            SDA_TRY(tmp.alloc((size_t)cnt * d));
            SDA_CUDA(cudaMemcpyAsync(tmp.p, o.rhs, (size_t)cnt * d * sizeof(double), cudaMemcpyHostToDevice, s));
            src = tmp.p;
        }
        SDA_TRY(permute_to_new(op, src, w.dev_b.p, cnt, s));
        SDA_CUDA(cudaStreamSynchronize(s));
    }
    int worst = SDA_OK;
    DevBuf<double> bt;
    if (o.batch_targets) {
        // right-hand side of every target of the call, then the batches
        std::vector<const double *> bl((size_t)tc);
        if (o.rhs_mode == SDA_RHS_FROM_R) SDA_TRY(bt.alloc((size_t)tc * d + 1));
        for (int i = 0; i < tc; ++i) {
            const int t = t0 + i;
            bl[(size_t)i] = op->dvec.p + (int64_t)t * d;
            if (o.rhs_mode == SDA_RHS_GIVEN) {
                bl[(size_t)i] = w.dev_b.p + (int64_t)i * d;
            } else if (o.rhs_mode == SDA_RHS_FROM_R) {
                const double *cnt = &op->counts[(size_t)t * 3];
                SDA_TRY(dot_f64(op, d, op->dvec.p + (int64_t)t * d, w.dev_b.p, bt.p + (int64_t)tc * d, s));
                k_scale<<<grid_elems(d, op->sm_count), kBlock, 0, s>>>(d, op->dvec.p + (int64_t)t * d,
                                                                      bt.p + (int64_t)tc * d, cnt[1] * cnt[2] / cnt[0],
                                                                      bt.p + (int64_t)i * d);
                SDA_LAUNCHED();
                bl[(size_t)i] = bt.p + (int64_t)i * d;
            }
        }
        SDA_TRY(solve_batched(op, t0, tc, bl.data(), shifts, n_shifts, o, alpha, omega, w_out, report, s, &worst));
    }
    if (o.rhs_mode == SDA_RHS_FROM_R && !o.batch_targets) SDA_TRY(bt.alloc((size_t)d + 1));
    for (int i = 0; i < (o.batch_targets ? 0 : tc); ++i) {
        const int t = t0 + i;
        const double *b = op->dvec.p + (int64_t)t * d;
        if (o.rhs_mode == SDA_RHS_GIVEN) {
            b = w.dev_b.p + (int64_t)i * d;
        } else if (o.rhs_mode == SDA_RHS_FROM_R) {
            // (X - 1 mu^T)^T [W 0; 0 0] X r = (N+ N- / l) (d^T r) d
            const double *cnt = &op->counts[(size_t)t * 3];
            SDA_TRY(dot_f64(op, d, op->dvec.p + (int64_t)t * d, w.dev_b.p, bt.p + d, s));
            k_scale<<<grid_elems(d, op->sm_count), kBlock, 0, s>>>(d, op->dvec.p + (int64_t)t * d, bt.p + d,
                                                                  cnt[1] * cnt[2] / cnt[0], bt.p);
            SDA_LAUNCHED();
            b = bt.p;
        }
        double *wt = w_out ? w_out + (int64_t)i * n_shifts * d : nullptr;
        sda_shift_report *rt = report ? report + (int64_t)i * n_shifts : nullptr;
        int rc;
        if (op->compute == SDA_F64) {
            rc = solve_target<double, double>(op, t, b, shifts, n_shifts, o, alpha, omega, wt, rt, s, &worst);
        } else {
            rc = with_vt(op->compute, [&](auto tag) -> int {
                using VT = std::remove_pointer_t<decltype(tag)>;
                return solve_target<VT, float>(op, t, b, shifts, n_shifts, o, alpha, omega, wt, rt, s, &worst);
            });
        }
        if (rc < 0) return rc;
    }
    if (op->stats.shift_form == 0) op->stats.shift_form = SDA_SHIFTS_RECURRENCE;
    SDA_CUDA(cudaEventRecord(w.call_ev[1], s));
    SDA_CUDA(cudaEventSynchronize(w.call_ev[1]));
    float call_ms = 0.f;
    SDA_CUDA(cudaEventElapsedTime(&call_ms, w.call_ev[0], w.call_ev[1]));
    op->stats.solve_ms = call_ms;
    return worst;
}

extern "C" SDA_API int sda_get_solve_stats(const sda_operator *op, sda_solve_stats *stats) {
    if (!op || !stats) return fail(SDA_ERR_INVALID_ARG, "NULL argument");
    *stats = op->stats;
    return SDA_OK;
}

extern "C" SDA_API int64_t sda_kernel_launch_count(void) { return launch_count(); }

// The contractions of the adjoint gradient of target t (FP64, permuted order):
// sc[1] = lambda^T w, sc[4] = (X~ lambda)^T L (X~ w), sc[5] = (X~ lambda)^T P_l (X~ w)
// (sc[2], sc[3]: mu^T w, mu^T lambda); uw, ul, v, v2: N-vector scratch.
static int adjoint_dots(const sda_operator *op, int t, const double *wp, const double *lam, double *uw, double *ul,
                        double *v, double *v2, double *sc, cudaStream_t s) {
    const int64_t d = op->d, n = op->n;
    const double *mu = op->mu.p + (int64_t)t * d;
    const int8_t *y = op->labels.p + (int64_t)t * n;
    SDA_TRY(dot_f64(op, d, lam, wp, sc + 1, s));
    SDA_TRY(dot_f64(op, d, mu, wp, sc + 2, s));
    SDA_TRY(dot_f64(op, d, mu, lam, sc + 3, s));
    SDA_TRY(op_xmul_f64(op, wp, uw, sc + 2, s));
    SDA_TRY(op_xmul_f64(op, lam, ul, sc + 3, s));
    SDA_TRY((rowpass<double, double>(op->s_lanes, n, op->s_rp.p, op->s_col.p, op->s_val64.p,
                                     GatherVec<double, double>{uw}, EpiLap64{v, uw, op->deg64.p, y, 0.0, 1.0},
                                     op->sm_count * kMaxBlocksPerSm, s)));
    SDA_TRY(dot_f64(op, n, ul, v, sc + 4, s));
    k_mask_labelled<<<grid_elems(n, op->sm_count), kBlock, 0, s>>>(n, y, uw, v2);
    SDA_LAUNCHED();
    SDA_TRY(dot_f64(op, n, ul, v2, sc + 5, s));
    return SDA_OK;
}

extern "C" SDA_API int sda_adjoint_grad(sda_operator *op, int32_t target, double alpha, double beta,
                                        const double *w, const double *dloss_ds, const int64_t *rows, int64_t n_rows,
                                        const sda_solve_opts *opt, double *d_alpha, double *d_beta,
                                        double *lambda_out, void *cuda_stream) {
    clear_error();
    if (!op || !w || !d_alpha || !d_beta) return fail(SDA_ERR_INVALID_ARG, "NULL argument");
    SDA_TRY(check_device(op->device));
    if (n_rows < 0 || (n_rows > 0 && (!rows || !dloss_ds))) return fail(SDA_ERR_INVALID_ARG, "bad held-out rows");
    if (target < 0 || target >= op->n_targets) return fail(SDA_ERR_INVALID_ARG, "target out of range");
    if (!(beta > 0.0) || !isfinite(beta)) return fail(SDA_ERR_INVALID_ARG, "beta must be finite and > 0");
    if (op->regression) return fail(SDA_ERR_UNSUPPORTED, "the adjoint is defined for SDA operators only");
    sda_solve_opts o;
    if (opt) {
        o = *opt;
    } else {
        sda_default_opts(&o);
        o.tol = 1e-10;
    }
    o.alpha = alpha;
    o.scatter_weight = NAN;
    o.rhs_mode = SDA_RHS_GIVEN;
    double al = 0.0, om = 0.0;
    SDA_TRY(call_weights(op, o, &al, &om));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    SDA_TRY(ensure_workspace(op, 1));
    Workspace &ws = op->ws;
    const int64_t d = op->d, n = op->n;
    if (ws.adj.n < (size_t)(3 * d + 5 * n)) SDA_TRY(ws.adj.alloc((size_t)(3 * d + 5 * n)));
    double *wp = ws.adj.p, *c = wp + d, *lam = c + d, *G = lam + d, *uw = G + n, *ul = uw + n, *v = ul + n;
    double *v2 = G;   // G is free once c is formed
    DevBuf<double> sc;
    DevBuf<int> err;
    SDA_TRY(sc.alloc(8));
    SDA_TRY(err.alloc(1));
    SDA_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    const double *mu = op->mu.p + (int64_t)target * d;
    const int8_t *y = op->labels.p + (int64_t)target * n;
    // right-hand side (X_h - 1 mu^T)^T g = X^T G - mu (1^T G), G = g scattered to the rows
    SDA_TRY(permute_to_new(op, w, wp, 1, s));
    SDA_CUDA(cudaMemsetAsync(G, 0, (size_t)n * sizeof(double), s));
    if (n_rows > 0) {
        k_scatter_rows<<<grid_elems(n_rows, op->sm_count), kBlock, 0, s>>>(n_rows, rows, dloss_ds, G, n, err.p);
        SDA_LAUNCHED();
    }
    SDA_TRY(op_xtmul_f64(op, G, c, s));
    SDA_TRY(dot_f64(op, n, G, nullptr, sc.p + 0, s));
    k_sub_mu<<<grid_elems(d, op->sm_count), kBlock, 0, s>>>(d, c, mu, sc.p + 0);
    SDA_LAUNCHED();
    int herr = 0;
    SDA_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    if (herr) return fail(SDA_ERR_INVALID_ARG, "a held-out row id is out of range");
    // adjoint solve (B + beta I) lambda = c on the same operator
    int worst = SDA_OK;
    sda_shift_report rep;
    int rc;
    if (op->compute == SDA_F64) {
        rc = solve_target<double, double>(op, target, c, &beta, 1, o, al, om, nullptr, &rep, s, &worst);
    } else {
        rc = with_vt(op->compute, [&](auto tag) -> int {
            using VT = std::remove_pointer_t<decltype(tag)>;
            return solve_target<VT, float>(op, target, c, &beta, 1, o, al, om, nullptr, &rep, s, &worst);
        });
    }
    if (rc < 0) return rc;
    // lambda: the solve's FP64 solution (permuted order)
    SDA_CUDA(cudaMemcpyAsync(lam, ws.w64.p, (size_t)d * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (worst < 0) return worst;
    SDA_TRY(adjoint_dots(op, target, wp, lam, uw, ul, v, v2, sc.p, s));
    if (lambda_out) SDA_TRY(permute_to_old(op, lam, lambda_out, 1, s));
    double hs[8];
    SDA_CUDA(cudaMemcpyAsync(hs, sc.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    *d_beta = -hs[1];
    *d_alpha = -(hs[4] - (op->omega_follows_alpha ? hs[5] : 0.0));
    return worst;
}

extern "C" SDA_API int sda_adjoint_grad_batched(sda_operator *op, int32_t n_targets, const int32_t *targets,
                                                double alpha, const double *betas, const double *W,
                                                const double *dloss_ds, const int64_t *rows, const int64_t *row_off,
                                                const sda_solve_opts *opt, double *d_alpha, double *d_beta,
                                                double *lambda_out, sda_shift_report *report, void *cuda_stream) {
    clear_error();
    if (!op || n_targets < 0) return fail(SDA_ERR_INVALID_ARG, "bad argument");
    SDA_TRY(check_device(op->device));
    if (op->regression) return fail(SDA_ERR_UNSUPPORTED, "the adjoint is defined for SDA operators only");
    if (n_targets == 0) return SDA_OK;
    if (!targets || !betas || !W || !row_off || !d_alpha || !d_beta) return fail(SDA_ERR_INVALID_ARG, "NULL argument");
    if (row_off[0] != 0) return fail(SDA_ERR_INVALID_ARG, "row_off[0] must be 0");
    for (int i = 0; i < n_targets; ++i) {
        if (targets[i] < 0 || targets[i] >= op->n_targets) return fail(SDA_ERR_INVALID_ARG, "target out of range");
        if (!(betas[i] > 0.0) || !isfinite(betas[i])) return fail(SDA_ERR_INVALID_ARG, "beta must be finite and > 0");
        if (row_off[i + 1] < row_off[i]) return fail(SDA_ERR_INVALID_ARG, "row_off must not decrease");
    }
    if (row_off[n_targets] > 0 && (!rows || !dloss_ds)) return fail(SDA_ERR_INVALID_ARG, "bad held-out rows");
    sda_solve_opts o;
    if (opt) {
        o = *opt;
    } else {
        sda_default_opts(&o);
        o.tol = 1e-10;
    }
    o.alpha = alpha;
    o.scatter_weight = NAN;
    o.rhs_mode = SDA_RHS_GIVEN;
    o.check_residual = 1;
    double al = 0.0, om = 0.0;
    SDA_TRY(call_weights(op, o, &al, &om));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t d = op->d, n = op->n, T = n_targets;
    DevBuf<double> wp, cb, lam, nv, sc;
    DevBuf<int> err;
    SDA_TRY(wp.alloc((size_t)(T * d)));
    SDA_TRY(cb.alloc((size_t)(T * d)));
    SDA_TRY(lam.alloc((size_t)(T * d)));
    const int64_t gl = std::min<int64_t>(T, 16);   // targets per FP64 block column pass
    SDA_TRY(nv.alloc((size_t)(gl * n)));
    SDA_TRY(sc.alloc((size_t)(8 * T)));
    SDA_TRY(err.alloc(1));
    SDA_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    SDA_TRY(permute_to_new(op, W, wp.p, T, s));
    // right-hand sides (X_h - 1 mu^T)^T g = X^T G - mu (1^T G), G = g scattered to the
    // held-out rows; X^T G of up to 16 targets per block column pass
    std::vector<const double *> bl((size_t)T);
    for (int64_t i0 = 0; i0 < T; i0 += gl) {
        const int nl = (int)std::min<int64_t>(gl, T - i0);
        const double *src[16];
        double *dst[16];
        SDA_CUDA(cudaMemsetAsync(nv.p, 0, (size_t)(nl * n) * sizeof(double), s));
        for (int k = 0; k < nl; ++k) {
            const int64_t i = i0 + k, r0 = row_off[i], nr = row_off[i + 1] - row_off[i];
            double *G = nv.p + (int64_t)k * n;   // g scattered to the held-out rows
            if (nr > 0) {
                k_scatter_rows<<<grid_elems(nr, op->sm_count), kBlock, 0, s>>>(nr, rows + r0, dloss_ds + r0, G, n,
                                                                              err.p);
                SDA_LAUNCHED();
            }
            src[k] = G;
            dst[k] = cb.p + i * d;
        }
        if (nl > 1) SDA_TRY(xt_lanes(op, src, nl, dst, s));
        else SDA_TRY(op_xtmul_f64(op, src[0], dst[0], s));
        for (int k = 0; k < nl; ++k) {
            const int64_t i = i0 + k;
            SDA_TRY(dot_f64(op, n, src[k], nullptr, sc.p + 8 * i, s));
            k_sub_mu<<<grid_elems(d, op->sm_count), kBlock, 0, s>>>(d, dst[k], op->mu.p + (int64_t)targets[i] * d,
                                                                   sc.p + 8 * i);
            SDA_LAUNCHED();
            bl[(size_t)i] = dst[k];
        }
    }
    int herr = 0;
    SDA_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    if (herr) return fail(SDA_ERR_INVALID_ARG, "a held-out row id is out of range");
    // the adjoint solves (B_t + beta_t I) lambda_t = c_t, 16 targets per batched run
    int worst = SDA_OK;
    memset(&op->stats, 0, sizeof(op->stats));
    SDA_TRY(solve_shift_lanes(op, targets, bl.data(), betas, n_targets, o, al, om, lam.p, report, s, &worst));
    if (worst < 0) return worst;
    // d/d beta = -lambda^T w (per target); the two cross terms of d/d alpha,
    // (X~ lambda)^T L (X~ w) and (X~ lambda)^T P_l (X~ w), 16 targets per FP64 block pass
    for (int64_t i = 0; i < T; ++i) SDA_TRY(dot_f64(op, d, lam.p + i * d, wp.p + i * d, sc.p + 8 * i + 1, s));
    std::vector<double> hs((size_t)(8 * T)), cross((size_t)(2 * T));
    for (int64_t i0 = 0; i0 < T; i0 += 16) {
        const int nl = (int)std::min<int64_t>(16, T - i0);
        SDA_TRY(adjoint_cross(op, targets + i0, nl, wp.p + i0 * d, lam.p + i0 * d, cross.data() + 2 * i0, s));
    }
    if (lambda_out) SDA_TRY(permute_to_old(op, lam.p, lambda_out, T, s));
    SDA_CUDA(cudaMemcpyAsync(hs.data(), sc.p, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < T; ++i) {
        d_beta[i] = -hs[(size_t)(8 * i + 1)];
        d_alpha[i] = -(cross[(size_t)(2 * i)] - (op->omega_follows_alpha ? cross[(size_t)(2 * i + 1)] : 0.0));
    }
    return worst;
}

extern "C" SDA_API int sda_operator_apply(const sda_operator *op, int32_t target, double sigma, const double *p,
                                          double *q, void *cuda_stream) {
    clear_error();
    if (!op || !p || !q) return fail(SDA_ERR_INVALID_ARG, "NULL argument");
    SDA_TRY(check_device(op->device));
    if (target < 0 || target >= op->n_targets) return fail(SDA_ERR_INVALID_ARG, "target out of range");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    sda_operator *mop = const_cast<sda_operator *>(op);
    SDA_TRY(ensure_apply_scratch(mop));
    double *pn = op->ws.f64.p, *qn = pn + op->d;
    SDA_TRY(permute_to_new(op, p, pn, 1, s));
    SDA_TRY(op_apply_f64(op, target, sigma, pn, qn, s, op->alpha, op->omega));
    SDA_TRY(permute_to_old(op, qn, q, 1, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    return SDA_OK;
}

extern "C" SDA_API int sda_project(const sda_operator *op, const double *w, int64_t n_vec, double *scores,
                                   int32_t centred, int32_t target, void *cuda_stream) {
    clear_error();
    if (!op || !w || !scores || n_vec < 0) return fail(SDA_ERR_INVALID_ARG, "bad argument");
    SDA_TRY(check_device(op->device));
    if (centred && (target < 0 || target >= op->n_targets)) return fail(SDA_ERR_INVALID_ARG, "target out of range");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    sda_operator *mop = const_cast<sda_operator *>(op);
    if (n_vec == 0) return SDA_OK;
    // the vectors in the permuted feature order, then X (or X~) on blocks of 16
    DevBuf<double> wn;
    SDA_TRY(wn.alloc((size_t)(n_vec * op->d)));
    SDA_TRY(permute_to_new(op, w, wn.p, n_vec, s));
    SDA_TRY(project_block(mop, wn.p, n_vec, scores, centred, target, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    return SDA_OK;
}

extern "C" SDA_API int sda_project_rows(const sda_operator *op, const double *w, int32_t n_vec, const int64_t *rows,
                                        int64_t n_rows, double *scores, int32_t centred, int32_t target,
                                        void *cuda_stream) {
    clear_error();
    if (!op || !w || !scores || n_vec < 0 || n_rows < 0 || (n_rows > 0 && !rows))
        return fail(SDA_ERR_INVALID_ARG, "bad argument");
    SDA_TRY(check_device(op->device));
    if (centred && (target < 0 || target >= op->n_targets)) return fail(SDA_ERR_INVALID_ARG, "target out of range");
    if (n_vec == 0 || n_rows == 0) return SDA_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t d = op->d;
    const int nb = std::min<int>(op->sm_count * 2, (int)((d + 31) / 32));
    // scratch in the operator's workspace (kept between calls, so repeated
    // calls allocate and free nothing): w permuted [n_vec][D], the centring
    // partials [nb][n_vec] and sums [n_vec], the row-id error flag
    const size_t b_wt = (size_t)n_vec * d * sizeof(double), b_part = (size_t)nb * n_vec * sizeof(double),
                 b_c = (size_t)n_vec * sizeof(double);
    const size_t need = b_wt + b_part + b_c + 256;
    sda_operator *mop = const_cast<sda_operator *>(op);
    if (mop->ws.proj.n < need) SDA_TRY(mop->ws.proj.alloc(need));
    double *wt = reinterpret_cast<double *>(mop->ws.proj.p), *part = wt + (size_t)n_vec * d,
           *c = part + (size_t)nb * n_vec;
    int *err = reinterpret_cast<int *>(c + n_vec);
    SDA_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    k_to_new_t<<<grid_elems(d * n_vec, op->sm_count), kBlock, 0, s>>>(d, n_vec, op->new_of_old.p, w, wt);
    SDA_LAUNCHED();
    if (centred) {
        k_mu_dots_part<<<nb, kBlock, 0, s>>>(d, n_vec, op->mu.p + (int64_t)target * d, wt, part);
        SDA_LAUNCHED();
        k_mu_dots_sum<<<(n_vec + 127) / 128, 128, 0, s>>>(nb, n_vec, part, c);
        SDA_LAUNCHED();
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n_rows + 7) / 8, (int64_t)op->sm_count * 16));
    SDA_TRY(with_vt(op->compute, [&](auto tag) -> int {
        using VT = std::remove_pointer_t<decltype(tag)>;
        k_project_rows<VT><<<grid, kBlock, 0, s>>>(op->n, n_rows, n_vec, rows, op->x_rp.p, op->x_col.p,
                                                   (const VT *)op->x_val_r.p, wt, centred ? c : nullptr, scores,
                                                   err);
        SDA_LAUNCHED();
        return SDA_OK;
    }));
    int herr = 0;
    SDA_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    if (herr) return fail(SDA_ERR_INVALID_ARG, "a row id is out of range");
    return SDA_OK;
}

extern "C" SDA_API int sda_get_operator_info(const sda_operator *op, sda_operator_info *info) {
    if (!op || !info) return fail(SDA_ERR_INVALID_ARG, "NULL argument");
    info->n_rows = op->n;
    info->n_cols = op->d;
    info->nnz = op->nnz;
    info->graph_nnz = op->s_nnz;
    info->n_targets = op->n_targets;
    info->compute = op->compute;
    info->alpha = op->alpha;
    info->omega = op->omega;
    info->device_bytes = op->bytes;
    info->col_ranges = op->xb.nranges;
    info->row_head = op->xr_head;
    info->col_entries = (int64_t)op->xb.idx.n;
    info->row_entries = (int64_t)op->xr_col.n;
    info->head_cols = (int32_t)op->hb.nseg;
    info->head_ranges = op->hb.nseg > 0 ? op->hb.nranges : 0;
    info->head_entries = op->hb.nseg > 0 ? (int64_t)op->hb.idx.n : 0;
    for (int k = 0; k < 4; ++k) info->tuned[k] = op->tuned[k];
    info->exact_x_passes = op->fx_state;
    info->x_frac_bits = (int16_t)(op->fx_state != 0 ? op->fx_sx : 0);
    info->x_int_bits = (int16_t)(op->fx_state != 0 ? op->fx_bx : 0);
    return SDA_OK;
}

extern "C" SDA_API int sda_get_target_counts(const sda_operator *op, double *counts) {
    if (!op || !counts) return fail(SDA_ERR_INVALID_ARG, "NULL argument");
    memcpy(counts, op->counts.data(), op->counts.size() * sizeof(double));
    return SDA_OK;
}

extern "C" SDA_API void sda_destroy_operator(sda_operator *op) {
    if (!op) return;
    // free on the operator's own device, then give the caller back theirs
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    const int dev = op->device;
    if (prev != dev) cudaSetDevice(dev);
    cudaDeviceSynchronize();
    release_workspace(op);
    release_batch(op);
    delete op;
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
}

extern "C" SDA_API const char *sda_status_string(int code) {
    switch (code) {
    case SDA_OK: return "SDA_OK";
    case SDA_NOT_CONVERGED: return "SDA_NOT_CONVERGED";
    case SDA_ERR_INVALID_ARG: return "SDA_ERR_INVALID_ARG";
    case SDA_ERR_SHAPE: return "SDA_ERR_SHAPE";
    case SDA_ERR_INDEX: return "SDA_ERR_INDEX";
    case SDA_ERR_VALUE_NOT_EXACT: return "SDA_ERR_VALUE_NOT_EXACT";
    case SDA_ERR_NO_POSITIVE: return "SDA_ERR_NO_POSITIVE";
    case SDA_ERR_NO_NEGATIVE: return "SDA_ERR_NO_NEGATIVE";
    case SDA_ERR_NOT_SYMMETRIC: return "SDA_ERR_NOT_SYMMETRIC";
    case SDA_ERR_BREAKDOWN: return "SDA_ERR_BREAKDOWN";
    case SDA_ERR_TIMEOUT: return "SDA_ERR_TIMEOUT";
    case SDA_ERR_CUDA: return "SDA_ERR_CUDA";
    case SDA_ERR_OOM: return "SDA_ERR_OOM";
    case SDA_ERR_UNSUPPORTED: return "SDA_ERR_UNSUPPORTED";
    default: return "SDA_UNKNOWN_STATUS";
    }
}

extern "C" SDA_API int sda_last_error_detail(char *buf, int len) { return last_error(buf, len); }
