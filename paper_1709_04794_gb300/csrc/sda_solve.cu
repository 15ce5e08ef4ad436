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
    __shared__ double red[kBlock / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock)
        s += b ? a[i] * b[i] : a[i];
    double mine[1] = {block_sum(s, red)};
    if (!arrive_last<1>(mine, partials, counter)) return;
    double tot[1];
    reduce_partials<1>(partials, gridDim.x, tot, red);
    if (threadIdx.x == 0) {
        *out = tot[0];
        *counter = 0u;
    }
}

// ||b - q||^2 into *out
__global__ void __launch_bounds__(kBlock) k_resid_f64(int64_t n, const double *__restrict__ b,
                                                      const double *__restrict__ q, double *out,
                                                      double *partials, unsigned *counter) {
    __shared__ double red[kBlock / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kBlock + threadIdx.x; i < n; i += (int64_t)gridDim.x * kBlock) {
        const double e = b[i] - q[i];
        s += e * e;
    }
    double mine[1] = {block_sum(s, red)};
    if (!arrive_last<1>(mine, partials, counter)) return;
    double tot[1];
    reduce_partials<1>(partials, gridDim.x, tot, red);
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
__global__ void k_w_out(int64_t d, int64_t ldw, int ns, const int32_t *new_of_old, const FT *W, double *out) {
    const int64_t m = d * ns;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i / d, o = i - s * d;
        out[i] = (double)W[s * ldw + new_of_old[o]];
    }
}

template <class FT>
__global__ void k_w_f64(int64_t d, const FT *W, double *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)W[i];
}

__global__ void k_scale(int64_t d, const double *x, const double *coef, double mult, double *out) {
    const double c = *coef * mult;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = c * x[i];
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

int op_xtmul_f64(const sda_operator *op, const double *v, double *q, cudaStream_t s) {
    return with_vt(op->compute, [&](auto tag) -> int {
        using VT = std::remove_pointer_t<decltype(tag)>;
        return segpass<VT, double>(op, op->col, 0, 0, op->x_cp.p, op->x_row.p, op->x_val_c.p,
                                   GatherVec<double, double>{v}, EpiStore<double>{q, nullptr, nullptr, 0.0}, op->grid,
                                   s);
    });
}

int op_xmul_f64(const sda_operator *op, const double *w, double *u, const double *csub, cudaStream_t s) {
    return with_vt(op->compute, [&](auto tag) -> int {
        using VT = std::remove_pointer_t<decltype(tag)>;
        return segpass<VT, double>(op, op->xrow, op->xrow_slot0, op->xrow_lseg0, op->x_rp.p, op->x_col.p,
                                   op->x_val_r.p, GatherVec<double, double>{w},
                                   EpiStore<double>{u, csub, nullptr, 0.0}, op->grid, s);
    });
}

static int dot_f64(const sda_operator *op, int64_t n, const double *a, const double *b, double *out, cudaStream_t s) {
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

// q = (B + sigma I) p, FP64, centred symmetric form, permuted order
int op_apply_f64(const sda_operator *op, int target, double sigma, const double *p, double *q, cudaStream_t s) {
    sda_operator *mop = const_cast<sda_operator *>(op);
    SDA_TRY(ensure_apply_scratch(mop));
    double *u = op->ws.f64.p + 3 * op->d, *v = u + op->n;
    const double *mu = op->mu.p + (int64_t)target * op->d;
    const int8_t *y = op->labels.p + (int64_t)target * op->n;
    SDA_TRY(dot_f64(op, op->d, mu, p, op->scal.p + 0, s));
    SDA_TRY(op_xmul_f64(op, p, u, op->scal.p + 0, s));
    SDA_TRY((segpass<double, double>(op, op->srow, op->srow_slot0, op->srow_lseg0, op->s_rp.p, op->s_col.p,
                                     op->s_val64.p, GatherVec<double, double>{u},
                                     EpiLap64{v, u, op->deg64.p, y, op->omega, op->alpha}, op->grid, s)));
    SDA_TRY(dot_f64(op, op->n, v, nullptr, op->scal.p + 1, s));
    return with_vt(op->compute, [&](auto tag) -> int {
        using VT = std::remove_pointer_t<decltype(tag)>;
        return segpass<VT, double>(op, op->col, 0, 0, op->x_cp.p, op->x_row.p, op->x_val_c.p,
                                   GatherVec<double, double>{v}, EpiApply{q, mu, p, op->scal.p + 1, sigma, 0.0},
                                   op->grid, s);
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
    w.dev_b.release();
}

static int ensure_workspace(sda_operator *op, int ns) {
    Workspace &w = op->ws;
    const int fp64 = op->compute == SDA_F64;
    const size_t fsz = fp64 ? sizeof(double) : sizeof(float);
    const int64_t ldw = (op->d + 7) / 8 * 8;
    const bool realloc = w.fp64 != fp64 || w.d != op->d || w.n != op->n || w.n_shifts < ns;
    if (!realloc) return SDA_OK;
    if (w.graph) cudaGraphExecDestroy(w.graph);
    w.graph = nullptr;
    w.graph_iters = 0;
    SDA_TRY(w.vec.alloc((size_t)(5 * ldw + 2 * op->n) * fsz));
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
    w.vt = -1;
    return SDA_OK;
}

template <class FT>
struct WsView {
    typename RPair<FT>::T *rp;
    FT *s, *ut, *v, *W, *P;
};

template <class FT>
static WsView<FT> view(const sda_operator *op) {
    const Workspace &w = op->ws;
    FT *base = (FT *)w.vec.p;
    FT *sb = (FT *)w.shift.p;
    const int64_t l = w.ldw;
    return WsView<FT>{(typename RPair<FT>::T *)base, base + 4 * l, base + 5 * l, base + 5 * l + op->n, sb,
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

template <class VT, class FT>
struct PhaseKernels {
    using K1 = GatherP<FT>;
    static constexpr auto p1 = k_segpass<VT, FT, GatherP<FT>, EpiP1<FT>>;
    static constexpr auto p2 = k_segpass<FT, FT, GatherVec<FT, FT>, EpiP2<FT>>;
    static constexpr auto p3a = k_segpass<VT, FT, GatherVec<FT, FT>, EpiStore<FT>>;
};

// sizes the grids of the iteration kernels for this operator's dtypes
template <class VT, class FT>
static int size_grids(sda_operator *op) {
    Workspace &w = op->ws;
    if (w.vt == (int)op->compute) return SDA_OK;
    const int sms = op->sm_count;
    w.grid1 = grid_of((const void *)PhaseKernels<VT, FT>::p1, sms);
    w.grid2 = grid_of((const void *)PhaseKernels<VT, FT>::p2, sms);
    w.grid3a = grid_of((const void *)PhaseKernels<VT, FT>::p3a, sms);
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
    const FT *sv = std::is_same<FT, double>::value ? (const FT *)op->s_val64.p : (const FT *)op->s_val32.p;
    const FT *dg = std::is_same<FT, double>::value ? (const FT *)op->deg64.p : (const FT *)op->deg32.p;
    const size_t P = (size_t)kMaxBlocksPerSm * op->sm_count;
    if (ev) SDA_CUDA(cudaEventRecord(ev[0], s));
    SDA_TRY((segpass<VT, FT>(op, op->xrow, op->xrow_slot0, op->xrow_lseg0, op->x_rp.p, op->x_col.p, op->x_val_r.p,
                             GatherP<FT>{b.rp, w.ldw, w.st.p, nullptr, (FT)0}, EpiP1<FT>{b.ut, w.st.p, 0.0}, w.grid1,
                             s)));
    if (ev) SDA_CUDA(cudaEventRecord(ev[1], s));
    if (ev) SDA_CUDA(cudaEventRecord(ev[2], s));
    SDA_TRY((segpass<FT, FT>(op, op->srow, op->srow_slot0, op->srow_lseg0, op->s_rp.p, op->s_col.p, sv,
                             GatherVec<FT, FT>{b.ut},
                             EpiP2<FT>{b.v, b.ut, dg, w.st.p, w.part.p + P * 4, w.cnt.p + 1, nullptr, 0, 0, 0, 0},
                             w.grid2, s)));
    if (ev) SDA_CUDA(cudaEventRecord(ev[3], s));
    if (ev) SDA_CUDA(cudaEventRecord(ev[4], s));
    SDA_TRY((segpass<VT, FT>(op, op->col, 0, 0, op->x_cp.p, op->x_row.p, op->x_val_c.p, GatherVec<FT, FT>{b.v},
                             EpiStore<FT>{b.s, nullptr, w.st.p, 0.0}, w.grid3a, s)));
    if (ev) SDA_CUDA(cudaEventRecord(ev[5], s));
    if (ev) SDA_CUDA(cudaEventRecord(ev[6], s));
    k_cg_phase3b<FT><<<w.grid3b, kBlock, 0, s>>>(op->d, w.ldw, b.s, b.rp, b.W, b.P, w.st.p, w.part.p + P * 8,
                                                 w.cnt.p + 2);
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

template <class VT, class FT>
static int solve_target(sda_operator *op, int t, const double *b_perm, const double *shifts, int ns,
                        const sda_solve_opts &o, double *w_out_t, sda_shift_report *rep_t, cudaStream_t s,
                        int *worst) {
    Workspace &w = op->ws;
    SDA_TRY((size_grids<VT, FT>(op)));
    WsView<FT> bv = view<FT>(op);
    SolveState &h = *w.h_st;
    memset(&h, 0, sizeof(SolveState));
    double sigma0 = shifts[0];
    for (int i = 1; i < ns; ++i) sigma0 = std::min(sigma0, shifts[i]);
    h.sigma0 = sigma0;
    h.omega = op->omega;
    h.alpha_l = op->alpha;
    h.tol = o.tol;
    h.n_shifts = ns;
    h.fixed = o.fixed_iters > 0 ? 1 : 0;
    h.limit = o.fixed_iters > 0 ? o.fixed_iters : o.max_iter;
    h.labels = op->labels.p + (int64_t)t * op->n;
    h.mu = op->mu.p + (int64_t)t * op->d;
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
    // solution out, in the caller's feature order
    if (w_out_t) {
        double *dst = w_out_t;
        double *tmp = nullptr;
        DevBuf<double> hostbuf;
        if (!o.out_on_device) {
            SDA_TRY(hostbuf.alloc((size_t)ns * op->d));
            tmp = hostbuf.p;
            dst = tmp;
        }
        k_w_out<FT><<<grid_elems((int64_t)ns * op->d, op->sm_count), kBlock, 0, s>>>(op->d, w.ldw, ns,
                                                                                      op->new_of_old.p, bv.W, dst);
        SDA_LAUNCHED();
        if (!o.out_on_device) {
            SDA_CUDA(cudaMemcpyAsync(w_out_t, tmp, (size_t)ns * op->d * sizeof(double), cudaMemcpyDeviceToHost, s));
            SDA_CUDA(cudaStreamSynchronize(s));
        }
    }
    // FP64 true residual of every shift
    std::vector<double> tres((size_t)ns, -1.0);
    if (o.check_residual) {
        double *w64 = w.f64.p, *q = w.f64.p + op->d;
        DevBuf<double> rs;
        SDA_TRY(rs.alloc((size_t)ns + 1));
        SDA_TRY(dot_f64(op, op->d, b_perm, b_perm, rs.p + ns, s));
        for (int i = 0; i < ns; ++i) {
            k_w_f64<FT><<<grid_elems(op->d, op->sm_count), kBlock, 0, s>>>(op->d, bv.W + (int64_t)i * w.ldw, w64);
            SDA_LAUNCHED();
            SDA_TRY(op_apply_f64(op, t, shifts[i], w64, q, s));
            k_resid_f64<<<op->grid, kBlock, 0, s>>>(op->d, b_perm, q, rs.p + i, op->part.p, op->cnt.p);
            SDA_LAUNCHED();
        }
        std::vector<double> hr((size_t)ns + 1);
        SDA_CUDA(cudaMemcpyAsync(hr.data(), rs.p, hr.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        SDA_CUDA(cudaStreamSynchronize(s));
        const double bn = sqrt(hr[ns]);
        for (int i = 0; i < ns; ++i) tres[i] = bn > 0 ? sqrt(hr[i]) / bn : sqrt(hr[i]);
    }
    op->stats.iterations += h.k;
    for (int i = 0; i < ns; ++i) op->stats.shift_iterations += h.sh[i].iters;
    for (int i = 0; i < ns; ++i) {
        const ShiftState &sh = h.sh[i];
        int st = SDA_OK;
        if (h.status != SDA_OK) st = h.status;
        else if (!h.fixed && sh.active) st = SDA_NOT_CONVERGED;
        if (st == SDA_NOT_CONVERGED && *worst == SDA_OK) *worst = SDA_NOT_CONVERGED;
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
}

extern "C" SDA_API int sda_solve_shifts(sda_operator *op, const double *shifts, int32_t n_shifts,
                                        const sda_solve_opts *opt, double *w_out, sda_shift_report *report,
                                        void *cuda_stream) {
    clear_error();
    if (!op || !shifts) return fail(SDA_ERR_INVALID_ARG, "operator and shifts must not be NULL");
    if (n_shifts < 1 || n_shifts > kMaxShifts) return fail(SDA_ERR_INVALID_ARG, "n_shifts must be in [1, %d]", kMaxShifts);
    for (int i = 0; i < n_shifts; ++i)
        if (!(shifts[i] > 0.0) || !isfinite(shifts[i])) return fail(SDA_ERR_INVALID_ARG, "shifts must be finite and > 0");
    sda_solve_opts o;
    if (opt) o = *opt;
    else sda_default_opts(&o);
    if (o.fixed_iters <= 0 && (!(o.tol >= 0.0) || o.max_iter < 0))
        return fail(SDA_ERR_INVALID_ARG, "tol must be >= 0 and max_iter >= 0");
    const int t0 = o.target_begin;
    const int tc = o.target_count < 0 ? op->n_targets - t0 : o.target_count;
    if (t0 < 0 || tc < 0 || t0 + tc > op->n_targets) return fail(SDA_ERR_INVALID_ARG, "target range out of bounds");
    if (o.rhs_mode != SDA_RHS_CANONICAL && !o.rhs) return fail(SDA_ERR_INVALID_ARG, "rhs is NULL");
    if (o.rhs_mode < 0 || o.rhs_mode > SDA_RHS_GIVEN) return fail(SDA_ERR_INVALID_ARG, "bad rhs_mode");
    cudaStream_t s = (cudaStream_t)cuda_stream;
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
    if (o.rhs_mode == SDA_RHS_FROM_R) SDA_TRY(bt.alloc((size_t)d + 1));
    for (int i = 0; i < tc; ++i) {
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
            rc = solve_target<double, double>(op, t, b, shifts, n_shifts, o, wt, rt, s, &worst);
        } else {
            rc = with_vt(op->compute, [&](auto tag) -> int {
                using VT = std::remove_pointer_t<decltype(tag)>;
                return solve_target<VT, float>(op, t, b, shifts, n_shifts, o, wt, rt, s, &worst);
            });
        }
        if (rc < 0) return rc;
    }
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

extern "C" SDA_API int sda_operator_apply(const sda_operator *op, int32_t target, double sigma, const double *p,
                                          double *q, void *cuda_stream) {
    clear_error();
    if (!op || !p || !q) return fail(SDA_ERR_INVALID_ARG, "NULL argument");
    if (target < 0 || target >= op->n_targets) return fail(SDA_ERR_INVALID_ARG, "target out of range");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    sda_operator *mop = const_cast<sda_operator *>(op);
    SDA_TRY(ensure_apply_scratch(mop));
    double *pn = op->ws.f64.p, *qn = pn + op->d;
    SDA_TRY(permute_to_new(op, p, pn, 1, s));
    SDA_TRY(op_apply_f64(op, target, sigma, pn, qn, s));
    SDA_TRY(permute_to_old(op, qn, q, 1, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    return SDA_OK;
}

extern "C" SDA_API int sda_project(const sda_operator *op, const double *w, int64_t n_vec, double *scores,
                                   int32_t centred, int32_t target, void *cuda_stream) {
    clear_error();
    if (!op || !w || !scores || n_vec < 0) return fail(SDA_ERR_INVALID_ARG, "bad argument");
    if (centred && (target < 0 || target >= op->n_targets)) return fail(SDA_ERR_INVALID_ARG, "target out of range");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    sda_operator *mop = const_cast<sda_operator *>(op);
    SDA_TRY(ensure_apply_scratch(mop));
    double *wn = op->ws.f64.p;
    for (int64_t v = 0; v < n_vec; ++v) {
        SDA_TRY(permute_to_new(op, w + v * op->d, wn, 1, s));
        const double *csub = nullptr;
        if (centred) {
            SDA_TRY(dot_f64(op, op->d, op->mu.p + (int64_t)target * op->d, wn, op->scal.p + 2, s));
            csub = op->scal.p + 2;
        }
        SDA_TRY(op_xmul_f64(op, wn, scores + v * op->n, csub, s));
    }
    SDA_CUDA(cudaStreamSynchronize(s));
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
    return SDA_OK;
}

extern "C" SDA_API int sda_get_target_counts(const sda_operator *op, double *counts) {
    if (!op || !counts) return fail(SDA_ERR_INVALID_ARG, "NULL argument");
    memcpy(counts, op->counts.data(), op->counts.size() * sizeof(double));
    return SDA_OK;
}

extern "C" SDA_API void sda_destroy_operator(sda_operator *op) {
    if (!op) return;
    cudaDeviceSynchronize();
    release_workspace(op);
    delete op;
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
