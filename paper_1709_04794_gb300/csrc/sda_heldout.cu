// sda_heldout_logistic: the held-out logistic loss of every (target, shift),
// the shift of least loss per target and the loss's derivative with respect
// to the ratings at that shift (the right-hand side data of the adjoint
// gradient).  The paper picks beta on held-out folds (Sec. 5); this is the
// selection step with the logistic loss as the criterion.
//
// Two launches per group of up to kHoTargets targets, the group's row offsets
// passed by value (no device allocation, no synchronisation):
//   k_heldout_loss  one block per (target, shift): a strided FP64 sum of
//                   softplus(-y s) per thread, then a fixed tree over the block
//   k_heldout_grad  one block per target: the least loss (first index on ties),
//                   then g over the target's rows at that shift
#include <math.h>

#include <algorithm>

#include "sda_common.cuh"

namespace sda {
namespace {

constexpr int kHoTargets = 256;   // targets per launch (their offsets travel by value)

struct HoOffsets {
    int64_t off[kHoTargets + 1];  // row_off[t0 .. t0 + nt] of the group starting at target t0
};

// log(1 + e^z) without overflow for large z
__device__ __forceinline__ double softplus(double z) {
    return z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z));
}

// 1 / (1 + e^m) without overflow for large |m|
__device__ __forceinline__ double inv_one_plus_exp(double m) {
    if (m >= 0.0) {
        const double e = exp(-m);
        return e / (1.0 + e);
    }
    return 1.0 / (1.0 + exp(m));
}

// fixed-order block sum (kBlock threads): the same bits on every call
__device__ double block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kBlock) k_heldout_loss(HoOffsets o, int ns, const double *__restrict__ scores,
                                                         const double *__restrict__ y, double *__restrict__ loss,
                                                         int t_base) {
    __shared__ double sh[kBlock];
    const int tl = blockIdx.x, s = blockIdx.y;
    const int64_t r0 = o.off[tl], m = o.off[tl + 1] - r0;
    const double *sc = scores + (int64_t)ns * r0 + (int64_t)s * m;
    double acc = 0.0;
    for (int64_t h = threadIdx.x; h < m; h += kBlock) acc += softplus(-y[r0 + h] * sc[h]);
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) loss[(int64_t)(t_base + tl) * ns + s] = m > 0 ? tot / (double)m : 0.0;
}

__global__ void __launch_bounds__(kBlock) k_heldout_grad(HoOffsets o, int ns, const double *__restrict__ scores,
                                                         const double *__restrict__ y,
                                                         const double *__restrict__ loss, int32_t *__restrict__ best,
                                                         double *__restrict__ g, int t_base) {
    __shared__ int s_best;
    const int tl = blockIdx.x;
    const int64_t r0 = o.off[tl], m = o.off[tl + 1] - r0;
    if (threadIdx.x == 0) {
        const double *lt = loss + (int64_t)(t_base + tl) * ns;
        int b = 0;
        double lb = lt[0];
        for (int s = 1; s < ns; ++s) {
            const double l = lt[s];
            if (isnan(lb) ? !isnan(l) : l < lb) {
                b = s;
                lb = l;
            }
        }
        s_best = b;
        best[t_base + tl] = b;
    }
    __syncthreads();
    const double *sc = scores + (int64_t)ns * r0 + (int64_t)s_best * m;
    for (int64_t h = threadIdx.x; h < m; h += kBlock) {
        const double yh = y[r0 + h];
        g[r0 + h] = -yh * inv_one_plus_exp(yh * sc[h]) / (double)m;
    }
}

}  // namespace
}  // namespace sda

using namespace sda;

extern "C" SDA_API int sda_heldout_logistic(int32_t n_targets, int32_t n_shifts, const int64_t *row_off,
                                            const double *scores, const double *y, double *loss, int32_t *best,
                                            double *g, void *cuda_stream) {
    clear_error();
    if (n_targets < 0 || n_shifts < 1 || !row_off) return fail(SDA_ERR_INVALID_ARG, "bad sizes");
    if (n_targets == 0) return SDA_OK;
    if (row_off[0] != 0) return fail(SDA_ERR_INVALID_ARG, "row_off[0] must be 0");
    for (int32_t t = 0; t < n_targets; ++t)
        if (row_off[t + 1] < row_off[t]) return fail(SDA_ERR_INVALID_ARG, "row_off decreases at target %d", t);
    const int64_t rows = row_off[n_targets];
    if (!loss || !best || (rows > 0 && (!scores || !y || !g))) return fail(SDA_ERR_INVALID_ARG, "a NULL array");
    if (n_shifts > 65535 || rows > INT64_MAX / n_shifts) return fail(SDA_ERR_INVALID_ARG, "too many shifts or rows");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    for (int32_t t0 = 0; t0 < n_targets; t0 += kHoTargets) {
        const int nt = std::min<int32_t>(kHoTargets, n_targets - t0);
        HoOffsets o;
        for (int i = 0; i <= nt; ++i) o.off[i] = row_off[t0 + i];
        k_heldout_loss<<<dim3(nt, n_shifts), kBlock, 0, s>>>(o, n_shifts, scores, y, loss, t0);
        SDA_LAUNCHED();
        k_heldout_grad<<<nt, kBlock, 0, s>>>(o, n_shifts, scores, y, loss, best, g, t0);
        SDA_LAUNCHED();
    }
    return SDA_OK;
}
