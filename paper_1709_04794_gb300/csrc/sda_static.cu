// sda_operator_apply_static: the FP64 operator apply q = (B + sigma I) p with
// all of its scratch in one file-scope device array, for callers that must not
// allocate device memory.  It launches the same kernels as sda_operator_apply
// and reads the operator's matrices; every per-call buffer (permuted p and q,
// the N-vectors u and v, reduction partials and counters, split-segment
// partial sums) lives in g_apply_scratch.
#include <math.h>
#include <string.h>

#include <mutex>
#include <type_traits>

#include "sda_kernels.cuh"

namespace sda {

// One array per device that loads the library, held until the process exits.
static __device__ __align__(256) double g_apply_scratch[SDA_STATIC_SCRATCH_DOUBLES];

constexpr int kMaxDevices = 64;
static double *g_scratch_addr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mu;

// Device address of g_apply_scratch on the current device (looked up once per
// device, with that device current; the host-side name is not a device address).
static int scratch_address(double **out) {
    int dev = 0;
    SDA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(SDA_ERR_UNSUPPORTED, "device ordinal %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        SDA_CUDA(cudaGetSymbolAddress(&p, g_apply_scratch));
        g_scratch_addr[dev] = (double *)p;
    }
    *out = g_scratch_addr[dev];
    return SDA_OK;
}

__global__ void k_static_to_new(int64_t d, const int32_t *new_of_old, const double *in, double *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
        out[new_of_old[i]] = in[i];
}

__global__ void k_static_to_old(int64_t d, const int32_t *new_of_old, const double *in, double *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[new_of_old[i]];
}

template <class VT, class Gather, class Epi>
static int static_pass(const sda_operator *op, const ColSchedule &sc, double *slots, unsigned *lcount,
                       const int64_t *ptr, const int32_t *idx, const void *val, const Gather &g, const Epi &e,
                       cudaStream_t s) {
    k_segpass<VT, double, Gather, Epi><<<op->grid, kBlock, 0, s>>>(sc.tiles.p, sc.ntiles, ptr, idx, (const VT *)val,
                                                                  g, e, slots, lcount, sc.splits.p);
    SDA_LAUNCHED();
    return SDA_OK;
}

template <class VT>
static int apply_static(const sda_operator *op, int32_t target, double sigma, const double *p, double *q,
                        double *scr, cudaStream_t s) {
    const int64_t n = op->n, d = op->d;
    const int nslots = op->col.nslots + op->xrow.nslots + op->srow.nslots;
    const int nsplits = op->col.nsplits + op->xrow.nsplits + op->srow.nsplits;
    // layout of the scratch, in doubles
    double *pn = scr, *qn = pn + d, *u = qn + d, *v = u + n;
    double *scal = v + n;                      // [0] <mu, p>, [1] 1^T v
    double *part = scal + 2;                   // block partials of the dot kernel
    double *slots = part + op->grid;           // split-segment partial sums
    unsigned *cnt = (unsigned *)(slots + nslots);   // [0] dot counter, [1..] split counters
    unsigned *lcount = cnt + 1;
    // counters must start at zero (a previous call leaves them at zero, but the
    // array is shared by every call and every operator)
    SDA_CUDA(cudaMemsetAsync(cnt, 0, (size_t)(1 + nsplits) * sizeof(unsigned), s));
    const int ge = (int)std::max<int64_t>(1, std::min<int64_t>((d + kBlock - 1) / kBlock, (int64_t)op->sm_count * 16));
    k_static_to_new<<<ge, kBlock, 0, s>>>(d, op->new_of_old.p, p, pn);
    SDA_LAUNCHED();
    const double *mu = op->mu.p + (int64_t)target * d;
    const int8_t *y = op->labels.p + (int64_t)target * n;
    k_dot_f64<<<op->grid, kBlock, 0, s>>>(d, mu, pn, scal + 0, part, cnt);
    SDA_LAUNCHED();
    SDA_TRY((static_pass<VT>(op, op->xrow, slots + op->xrow_slot0, lcount + op->xrow_lseg0, op->x_rp.p, op->x_col.p,
                             op->x_val_r.p, GatherVec<double, double>{pn}, EpiStore<double>{u, scal + 0, nullptr, 0.0},
                             s)));
    SDA_TRY((static_pass<double>(op, op->srow, slots + op->srow_slot0, lcount + op->srow_lseg0, op->s_rp.p,
                                 op->s_col.p, op->s_val64.p, GatherVec<double, double>{u},
                                 EpiLap64{v, u, op->deg64.p, y, op->omega, op->alpha}, s)));
    k_dot_f64<<<op->grid, kBlock, 0, s>>>(n, v, nullptr, scal + 1, part, cnt);
    SDA_LAUNCHED();
    SDA_TRY((static_pass<VT>(op, op->col, slots, lcount, op->x_cp.p, op->x_row.p, op->x_val_c.p,
                             GatherVec<double, double>{v}, EpiApply{qn, mu, pn, scal + 1, sigma, 0.0}, s)));
    k_static_to_old<<<ge, kBlock, 0, s>>>(d, op->new_of_old.p, qn, q);
    SDA_LAUNCHED();
    return SDA_OK;
}

}  // namespace sda

using namespace sda;

extern "C" SDA_API int sda_operator_apply_static(const sda_operator *op, int32_t target, double sigma,
                                                 const double *p, double *q, void *cuda_stream) {
    clear_error();
    if (!op || !p || !q) return fail(SDA_ERR_INVALID_ARG, "NULL argument");
    SDA_TRY(check_device(op->device));
    if (target < 0 || target >= op->n_targets) return fail(SDA_ERR_INVALID_ARG, "target out of range");
    const int64_t nslots = (int64_t)op->col.nslots + op->xrow.nslots + op->srow.nslots;
    const int64_t nsplits = (int64_t)op->col.nsplits + op->xrow.nsplits + op->srow.nsplits;
    const int64_t need = 2 * op->d + 2 * op->n + 2 + op->grid + nslots + (1 + nsplits + 1) / 2;
    if (need > (int64_t)SDA_STATIC_SCRATCH_DOUBLES)
        return fail(SDA_ERR_SHAPE,
                    "operator too large for the static scratch: needs %lld doubles (2 D + 2 N + %lld), "
                    "the array holds %lld",
                    (long long)need, (long long)(need - 2 * op->d - 2 * op->n), (long long)SDA_STATIC_SCRATCH_DOUBLES);
    double *scr = nullptr;
    SDA_TRY(scratch_address(&scr));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    switch (op->compute) {
    case SDA_F64: return apply_static<double>(op, target, sigma, p, q, scr, s);
    case SDA_F32: return apply_static<float>(op, target, sigma, p, q, scr, s);
    case SDA_F16: return apply_static<__half>(op, target, sigma, p, q, scr, s);
    case SDA_F8E4M3: return apply_static<__nv_fp8_e4m3>(op, target, sigma, p, q, scr, s);
    case SDA_PATTERN: return apply_static<Pattern>(op, target, sigma, p, q, scr, s);
    default: return fail(SDA_ERR_INVALID_ARG, "bad compute dtype");
    }
}
