// Device kernels of the operator apply and of the shifted-CG iteration.
//
// One iteration of Algorithm 3 on the centred operator
//   (B + sigma0 I) p = (X - 1 mu^T)^T M (X - 1 mu^T) p + sigma0 p,
//   M = omega P_l + alpha L,  L = D - S                        (eq. 7, Alg. 7, Sec. 3.2.3)
// runs as three passes over the data, each a single kernel:
//   phase 1 (rows of X):    ut = X p_k - <mu, p_k> 1            (p_k = r_k + alpha_k p_{k-1} formed on the fly)
//   phase 2 (rows of S):    v = omega P_l ut + alpha (D ut - S ut);  <ut, v>, 1^T v
//                           -> gamma_k, zeta^s_{k+1}, gamma^s_k
//   phase 3 (columns of X): q = X^T v - mu (1^T v) + sigma0 p_k;  r_{k+1} = r_k + gamma_k q;
//                           P^s_k = zeta^s_k r_k + alpha^s_k P^s_{k-1};  W^s_{k+1} = W^s_k - gamma^s_k P^s_k;
//                           <r,r>, <mu,r>, <r,p_k>  -> alpha_{k+1}, <mu,p_{k+1}>, <p_{k+1},p_{k+1}>, stop tests
// <p, (B + sigma0) p> = <ut, v> + sigma0 <p, p> is known after phase 2, so q is
// never stored; <mu, p> and <p, p> follow from recurrences on the phase-3 dots.
// The scalar work of a phase runs in the block that finishes last.
#pragma once

#include "sda_operator.cuh"

namespace sda {

template <class FT>
__device__ __forceinline__ FT form_p(FT r, FT p, FT a);
template <>
__device__ __forceinline__ float form_p<float>(float r, float p, float a) { return fmaf(a, p, r); }
template <>
__device__ __forceinline__ double form_p<double>(double r, double p, double a) { return fma(a, p, r); }

// ---------------------------------------------------------------------------
// column tile: column sums of X^T v, handed to an epilogue
// ---------------------------------------------------------------------------
// Epi must provide
//   __device__ void column(int64_t j, AccT sum)      one thread per column, consecutive columns on
//                                                    consecutive threads
//   __device__ void column_block(int64_t j, AccT s)  the whole block, one column (s valid in all threads)
template <class VT, class AccT, class Epi>
__device__ __forceinline__ void col_tile(const Tile &tl, const int64_t *__restrict__ cp,
                                         const int32_t *__restrict__ row, const VT *__restrict__ val,
                                         const AccT *__restrict__ v, AccT *slots, unsigned *lcount,
                                         const SplitSeg *__restrict__ splits, Epi &epi, AccT *qs,
                                         AccT *red) {
    __shared__ int s_last;
    if (tl.lanes > 0) {
        const int G = tl.lanes, ngroups = kBlock / G;
        const int g = threadIdx.x / G, lane = threadIdx.x % G;
        const int nseg = tl.seg1 - tl.seg0;
        for (int base = 0; base < nseg; base += ngroups) {
            const int s = base + g;
            AccT acc = 0;
            if (s < nseg) {
                const int64_t j = tl.seg0 + s;
                const int64_t e1 = cp[j + 1];
                for (int64_t e = cp[j] + lane; e < e1; e += G)
                    acc += (AccT)Val<VT>::get(val, e) * v[row[e]];
            }
            for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (s < nseg && lane == 0) qs[s] = acc;
        }
        __syncthreads();
        for (int s = threadIdx.x; s < nseg; s += kBlock) epi.column(tl.seg0 + s, qs[s]);
        __syncthreads();
        return;
    }
    AccT acc = 0;
    for (int64_t e = tl.nz0 + threadIdx.x; e < tl.nz1; e += kBlock)
        acc += (AccT)Val<VT>::get(val, e) * v[row[e]];
    acc = block_sum(acc, red);
    if (tl.slot < 0) {
        epi.column_block(tl.seg0, acc);
        return;
    }
    // one chunk of a split column: the chunk that completes it finishes the column
    if (threadIdx.x == 0) {
        slots[tl.slot] = acc;
        __threadfence();
        const unsigned prev = atomicAdd(&lcount[tl.lseg], 1u);
        s_last = (prev == (unsigned)splits[tl.lseg].nchunks - 1u);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        const SplitSeg sp = splits[tl.lseg];
        AccT tot = 0;
        for (int c = 0; c < sp.nchunks; ++c) tot += __ldcg(slots + sp.slot0 + c);   // fixed order
        if (threadIdx.x == 0) lcount[tl.lseg] = 0u;
        epi.column_block(tl.seg0, tot);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// plain FP64 kernels (operator apply, means, projection, residual check)
// ---------------------------------------------------------------------------

// u_i = sum_e x_e w[col_e] - (csub ? *csub : 0), groups of G lanes per row
template <class VT, int G>
__global__ void __launch_bounds__(kBlock) k_rows_f64(int64_t n, const int64_t *__restrict__ rp,
                                                     const int32_t *__restrict__ col,
                                                     const VT *__restrict__ val,
                                                     const double *__restrict__ w, double *__restrict__ u,
                                                     const double *csub) {
    constexpr int RPW = 32 / G;
    const double c = csub ? *csub : 0.0;
    const int lane = threadIdx.x % G;
    const int64_t warp = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kBlock) >> 5;
    for (int64_t base = warp * RPW; base < n; base += nwarps * RPW) {
        const int64_t i = base + (threadIdx.x & 31) / G;
        double acc = 0.0;
        if (i < n) {
            const int64_t e1 = rp[i + 1];
            for (int64_t e = rp[i] + lane; e < e1; e += G) acc += (double)Val<VT>::get(val, e) * w[col[e]];
        }
#pragma unroll
        for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < n && lane == 0) u[i] = acc - c;
    }
}

// v_i = omega [y_i != 0] ut_i + alpha (deg_i ut_i - sum_j s_ij ut_j)
template <int G>
__global__ void __launch_bounds__(kBlock) k_lap_f64(int64_t n, const int64_t *__restrict__ rp,
                                                    const int32_t *__restrict__ col,
                                                    const double *__restrict__ sv,
                                                    const double *__restrict__ deg,
                                                    const int8_t *__restrict__ y, double omega, double alpha,
                                                    const double *__restrict__ ut, double *__restrict__ v) {
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x % G;
    const int64_t warp = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kBlock) >> 5;
    for (int64_t base = warp * RPW; base < n; base += nwarps * RPW) {
        const int64_t i = base + (threadIdx.x & 31) / G;
        double acc = 0.0;
        if (i < n) {
            const int64_t e1 = rp[i + 1];
            for (int64_t e = rp[i] + lane; e < e1; e += G) acc += sv[e] * ut[col[e]];
        }
#pragma unroll
        for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < n && lane == 0) {
            const double u = ut[i];
            v[i] = omega * (y[i] != 0 ? u : 0.0) + alpha * (deg[i] * u - acc);
        }
    }
}

// <a, b> (or sum of a when b is NULL) into *out, fixed-order reduction
__global__ void __launch_bounds__(kBlock) k_dot_f64(int64_t n, const double *__restrict__ a,
                                                    const double *__restrict__ b, double *out,
                                                    double *partials, unsigned *counter);

struct EpiStore {
    double *q;
    __device__ __forceinline__ void column(int64_t j, double s) { q[j] = s; }
    __device__ __forceinline__ void column_block(int64_t j, double s) {
        if (threadIdx.x == 0) q[j] = s;
    }
};

// q_j = s_j - mu_j t + sigma p_j
struct EpiApply {
    double *q;
    const double *mu, *p;
    const double *t;
    double sigma;
    __device__ __forceinline__ void column(int64_t j, double s) { q[j] = s - mu[j] * (*t) + sigma * p[j]; }
    __device__ __forceinline__ void column_block(int64_t j, double s) {
        if (threadIdx.x == 0) column(j, s);
    }
};

template <class VT, class Epi>
__global__ void __launch_bounds__(kBlock) k_cols_f64(const Tile *__restrict__ tiles, int ntiles,
                                                     const int64_t *__restrict__ cp,
                                                     const int32_t *__restrict__ row,
                                                     const VT *__restrict__ val, const double *__restrict__ v,
                                                     double *slots, unsigned *lcount,
                                                     const SplitSeg *__restrict__ splits, Epi epi) {
    __shared__ double qs[kTileSegs];
    __shared__ double red[kBlock / 32];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        col_tile<VT, double, Epi>(tl, cp, row, val, v, slots, lcount, splits, epi, qs, red);
    }
}

// ---------------------------------------------------------------------------
// shifted CG (Algorithm 3) phase kernels; FT = vector type (float or double)
// ---------------------------------------------------------------------------

// r = b, p_{-1} = 0, W = 0, P_{-1} = 0; <r,r>, <mu,r>; scalar start values.
template <class FT>
__global__ void __launch_bounds__(kBlock) k_cg_init(int64_t d, const double *__restrict__ b, FT *r, FT *p,
                                                    FT *W, FT *P, SolveState *st, double *partials,
                                                    unsigned *counter) {
    __shared__ double red[kBlock / 32];
    const int ns = st->n_shifts;
    const double *mu = st->mu;
    double d0 = 0.0, d1 = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x; j < d; j += (int64_t)gridDim.x * kBlock) {
        const FT rj = (FT)b[j];
        r[j] = rj;
        p[j] = (FT)0;
        for (int s = 0; s < ns; ++s) {
            W[(int64_t)s * d + j] = (FT)0;
            P[(int64_t)s * d + j] = (FT)0;
        }
        d0 += (double)rj * (double)rj;
        d1 += mu[j] * (double)rj;
    }
    double mine[2];
    mine[0] = block_sum(d0, red);
    mine[1] = block_sum(d1, red);
    if (!arrive_last<2>(mine, partials, counter)) return;
    double tot[2];
    reduce_partials<2>(partials, gridDim.x, tot, red);
    if (threadIdx.x == 0) {
        st->rr = tot[0];
        st->bnorm = sqrt(tot[0]);
        st->c = tot[1];
        st->pp = tot[0];
        st->alpha = 0.0;
        st->gamma = 0.0;
        st->gamma_prev = 1.0;
        st->t = 0.0;
        st->k = 0;
        st->status = SDA_OK;
        *counter = 0u;
    }
    __syncthreads();
    const bool zero_rhs = !(st->bnorm > 0.0);
    for (int s = threadIdx.x; s < ns; s += kBlock) {
        ShiftState &h = st->sh[s];
        h.z_prev = 1.0;
        h.z = 1.0;
        h.z_next = 1.0;
        h.g = 0.0;
        h.a = 0.0;
        h.res = zero_rhs ? 0.0 : 1.0;
        h.active = (zero_rhs && !st->fixed) ? 0 : 1;
        h.iters = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int na = 0;
        for (int s = 0; s < ns; ++s) na += st->sh[s].active;
        st->nactive = na;
        st->done = (na == 0 || st->limit <= 0) ? 1 : 0;
    }
}

// phase 1: ut = X (r + alpha_k p) - c_k
template <class VT, class FT, int G>
__global__ void __launch_bounds__(kBlock) k_cg_phase1(int64_t n, const int64_t *__restrict__ rp,
                                                      const int32_t *__restrict__ col,
                                                      const VT *__restrict__ val, const FT *__restrict__ r,
                                                      const FT *__restrict__ p, FT *__restrict__ ut,
                                                      const SolveState *__restrict__ st) {
    if (st->done) return;
    const FT a = (FT)st->alpha;
    const double c = st->c;
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x % G;
    const int64_t warp = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kBlock) >> 5;
    for (int64_t base = warp * RPW; base < n; base += nwarps * RPW) {
        const int64_t i = base + (threadIdx.x & 31) / G;
        FT acc = 0;
        if (i < n) {
            const int64_t e1 = rp[i + 1];
            for (int64_t e = rp[i] + lane; e < e1; e += G) {
                const int32_t j = col[e];
                acc += (FT)Val<VT>::get(val, e) * form_p<FT>(r[j], p[j], a);
            }
        }
#pragma unroll
        for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < n && lane == 0) ut[i] = (FT)((double)acc - c);
    }
}

// phase 2: v = omega P_l ut + alpha (D ut - S ut); dots <ut,v>, 1^T v; then gamma_k and zeta^s_{k+1}
template <class FT, int G>
__global__ void __launch_bounds__(kBlock) k_cg_phase2(int64_t n, const int64_t *__restrict__ rp,
                                                      const int32_t *__restrict__ col,
                                                      const FT *__restrict__ sv, const FT *__restrict__ deg,
                                                      const FT *__restrict__ ut, FT *__restrict__ v,
                                                      SolveState *st, double *partials, unsigned *counter) {
    __shared__ double red[kBlock / 32];
    if (st->done) return;
    const int8_t *__restrict__ y = st->labels;
    const double omega = st->omega, al = st->alpha_l;
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x % G;
    const int64_t warp = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kBlock) >> 5;
    double d0 = 0.0, d1 = 0.0;
    for (int64_t base = warp * RPW; base < n; base += nwarps * RPW) {
        const int64_t i = base + (threadIdx.x & 31) / G;
        FT acc = 0;
        if (i < n) {
            const int64_t e1 = rp[i + 1];
            for (int64_t e = rp[i] + lane; e < e1; e += G) acc += sv[e] * ut[col[e]];
        }
#pragma unroll
        for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < n && lane == 0) {
            const double u = (double)ut[i];
            const double vi = omega * (y[i] != 0 ? u : 0.0) + al * ((double)deg[i] * u - (double)acc);
            const FT vf = (FT)vi;
            v[i] = vf;
            d0 += u * (double)vf;
            d1 += (double)vf;
        }
    }
    double mine[2];
    mine[0] = block_sum(d0, red);
    mine[1] = block_sum(d1, red);
    if (!arrive_last<2>(mine, partials, counter)) return;
    double tot[2];
    reduce_partials<2>(partials, gridDim.x, tot, red);
    if (threadIdx.x == 0) {
        const double pq = tot[0] + st->sigma0 * st->pp;
        if (!(pq > 0.0) || !isfinite(pq)) {
            st->status = SDA_ERR_BREAKDOWN;
            st->done = 1;
        } else {
            st->gamma = -st->rr / pq;
            st->t = tot[1];
        }
        *counter = 0u;
    }
    __syncthreads();
    if (st->status != SDA_OK) return;
    const double gam = st->gamma, gp = st->gamma_prev, al_k = st->alpha;
    for (int s = threadIdx.x; s < st->n_shifts; s += kBlock) {
        ShiftState &h = st->sh[s];
        if (!h.active) continue;
        const double den = gam * al_k * (h.z_prev - h.z) + h.z_prev * gp * (1.0 - h.delta * gam);
        const double zn = h.z_prev * h.z * gp / den;
        h.z_next = zn;
        h.g = gam * zn / h.z;
    }
}

// block-cached scalars of phase 3
template <class FT>
struct P3Shared {
    double alpha, gamma, t, sigma0;
    int nact;
    int act[kMaxShifts];
    FT zk[kMaxShifts], ak[kMaxShifts], gk[kMaxShifts];
    FT rb;   // r_k,j of a whole-block column
};

template <class FT>
struct EpiCG3 {
    FT *__restrict__ r;
    FT *__restrict__ p;
    FT *__restrict__ W;
    FT *__restrict__ P;
    const double *__restrict__ mu;
    int64_t d;
    P3Shared<FT> *sm;
    double dot[3];   // <r_{k+1}, r_{k+1}>, <mu, r_{k+1}>, <r_{k+1}, p_k>

    // scalar part of a column; returns r_k,j
    __device__ __forceinline__ FT scalar_part(int64_t j, double s) {
        const FT rj = r[j];
        const FT pk = form_p<FT>(rj, p[j], (FT)sm->alpha);
        const double mj = mu[j];
        const double q = s - mj * sm->t + sm->sigma0 * (double)pk;
        const FT rn = (FT)((double)rj + sm->gamma * q);
        r[j] = rn;
        p[j] = pk;
        dot[0] += (double)rn * (double)rn;
        dot[1] += mj * (double)rn;
        dot[2] += (double)rn * (double)pk;
        return rj;
    }
    __device__ __forceinline__ void shift_part(int64_t j, FT rj, int a) {
        const int s = sm->act[a];
        FT *Ps = P + (int64_t)s * d;
        FT *Ws = W + (int64_t)s * d;
        const FT pn = sm->zk[a] * rj + sm->ak[a] * Ps[j];
        Ps[j] = pn;
        Ws[j] -= sm->gk[a] * pn;
    }
    template <class AccT>
    __device__ __forceinline__ void column(int64_t j, AccT s) {
        const FT rj = scalar_part(j, (double)s);
        const int na = sm->nact;
        for (int a = 0; a < na; ++a) shift_part(j, rj, a);
    }
    template <class AccT>
    __device__ __forceinline__ void column_block(int64_t j, AccT s) {
        if (threadIdx.x == 0) sm->rb = scalar_part(j, (double)s);
        __syncthreads();
        const FT rj = sm->rb;
        for (int a = threadIdx.x; a < sm->nact; a += kBlock) shift_part(j, rj, a);
        __syncthreads();
    }
};

// phase 3: q = X^T v - mu t + sigma0 p_k; r, p, W, P updates; dots; then alpha_{k+1} and stop tests
template <class VT, class FT>
__global__ void __launch_bounds__(kBlock) k_cg_phase3(const Tile *__restrict__ tiles, int ntiles,
                                                      const int64_t *__restrict__ cp,
                                                      const int32_t *__restrict__ row,
                                                      const VT *__restrict__ val, const FT *__restrict__ v,
                                                      FT *r, FT *p, FT *W, FT *P, int64_t d, SolveState *st,
                                                      double *partials, unsigned *counter, FT *slots,
                                                      unsigned *lcount, const SplitSeg *__restrict__ splits) {
    __shared__ FT qs[kTileSegs];
    __shared__ FT redf[kBlock / 32];
    __shared__ double red[kBlock / 32];
    __shared__ P3Shared<FT> sm;
    if (st->done) return;
    if (threadIdx.x == 0) {
        sm.alpha = st->alpha;
        sm.gamma = st->gamma;
        sm.t = st->t;
        sm.sigma0 = st->sigma0;
        int na = 0;
        for (int s = 0; s < st->n_shifts; ++s) {
            const ShiftState &h = st->sh[s];
            if (!h.active) continue;
            sm.act[na] = s;
            sm.zk[na] = (FT)h.z;
            sm.ak[na] = (FT)h.a;
            sm.gk[na] = (FT)h.g;
            ++na;
        }
        sm.nact = na;
    }
    __syncthreads();
    EpiCG3<FT> epi{r, p, W, P, st->mu, d, &sm, {0.0, 0.0, 0.0}};
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        col_tile<VT, FT, EpiCG3<FT>>(tl, cp, row, val, v, slots, lcount, splits, epi, qs, redf);
    }
    double mine[3];
    mine[0] = block_sum(epi.dot[0], red);
    mine[1] = block_sum(epi.dot[1], red);
    mine[2] = block_sum(epi.dot[2], red);
    if (!arrive_last<3>(mine, partials, counter)) return;
    double tot[3];
    reduce_partials<3>(partials, gridDim.x, tot, red);
    __shared__ double s_alpha_new, s_rnorm;
    if (threadIdx.x == 0) {
        const double rr_new = tot[0];
        const double an = rr_new / st->rr;
        const double c_new = tot[1] + an * st->c;
        const double pp_new = rr_new + 2.0 * an * tot[2] + an * an * st->pp;
        if (!isfinite(rr_new) || !isfinite(an)) {
            st->status = SDA_ERR_BREAKDOWN;
        }
        st->gamma_prev = st->gamma;
        st->alpha = an;
        st->c = c_new;
        st->pp = pp_new;
        st->rr = rr_new;
        st->k = st->k + 1;
        s_alpha_new = an;
        s_rnorm = sqrt(rr_new);
        *counter = 0u;
    }
    __syncthreads();
    const double an = s_alpha_new, rnorm = s_rnorm, bnorm = st->bnorm, tol = st->tol;
    const int k = st->k, fixed = st->fixed;
    for (int s = threadIdx.x; s < st->n_shifts; s += kBlock) {
        ShiftState &h = st->sh[s];
        if (!h.active) continue;
        const double ratio = h.z_next / h.z;
        h.a = an * ratio * ratio;
        h.z_prev = h.z;
        h.z = h.z_next;
        h.iters = k;
        const double rz = fabs(h.z) * rnorm;
        h.res = bnorm > 0.0 ? rz / bnorm : 0.0;
        if (!fixed && (rz < tol * bnorm || !(fabs(h.z) > 0.0))) h.active = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int na = 0;
        for (int s = 0; s < st->n_shifts; ++s) na += st->sh[s].active;
        st->nactive = na;
        st->done = (na == 0 || k >= st->limit || st->status != SDA_OK) ? 1 : 0;
    }
}

}  // namespace sda
