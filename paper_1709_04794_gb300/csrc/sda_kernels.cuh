// Device kernels of the operator apply and of the shifted-CG iteration.
//
// One iteration of Algorithm 3 on the centred operator
//   (B + sigma0 I) p = (X - 1 mu^T)^T M (X - 1 mu^T) p + sigma0 p,
//   M = omega P_l + alpha L,  L = D - S                        (eq. 7, Alg. 7, Sec. 3.2.3)
// runs as four kernels:
//   phase 1  (rows of X):     ut = X p_k - <mu, p_k> 1   (p_k = r_k + alpha_k p_{k-1} formed at the gather)
//   phase 2  (rows of S):     v = omega P_l ut + alpha (D ut - S ut);  <ut, v>, 1^T v
//                             -> gamma_k, zeta^s_{k+1}, gamma^s_k
//   phase 3a (columns of X):  s = X^T v
//   phase 3b (stream over D): q = s - mu (1^T v) + sigma0 p_k;  r_{k+1} = r_k + gamma_k q;
//                             P^s_k = zeta^s_k r_k + alpha^s_k P^s_{k-1};  W^s_{k+1} = W^s_k - gamma^s_k P^s_k;
//                             <r,r>, <mu,r>, <r,p_k>  -> alpha_{k+1}, <mu,p_{k+1}>, <p_{k+1},p_{k+1}>, stop tests
// <p, (B + sigma0) p> = <ut, v> + sigma0 <p, p> is known after phase 2, so q is
// never stored; <mu, p> and <p, p> follow from recurrences on the phase-3b dots.
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
// `buf` holds kTileNnz AccT (shared).  Three tile kinds:
//   lanes < 0  short columns: the tile's nonzeros are loaded and multiplied with
//              all loads independent (coalesced index/value streams, gathers of v
//              in flight together), products staged in shared memory, then summed
//              per column in index order;
//   lanes > 0  a group of `lanes` lanes per column, xor-tree sum inside the group;
//   lanes == 0 one column or one chunk of a long column for the whole block; the
//              chunks of a split column leave their sums in slots and the chunk
//              that arrives last adds them in chunk order.
template <class VT, class AccT, class Epi>
__device__ __forceinline__ void col_tile(const Tile &tl, const int64_t *__restrict__ cp,
                                         const int32_t *__restrict__ row, const VT *__restrict__ val,
                                         const AccT *__restrict__ v, AccT *slots, unsigned *lcount,
                                         const SplitSeg *__restrict__ splits, Epi &epi, AccT *buf,
                                         AccT *red) {
    __shared__ int s_last;
    if (tl.lanes < 0) {
        const int64_t nz0 = tl.nz0;
        const int nnz = (int)(tl.nz1 - nz0);
        for (int e = threadIdx.x; e < nnz; e += kBlock)
            buf[e] = (AccT)Val<VT>::get(val, nz0 + e) * v[row[nz0 + e]];
        __syncthreads();
        const int nseg = tl.seg1 - tl.seg0;
        for (int s = threadIdx.x; s < nseg; s += kBlock) {
            const int64_t j = tl.seg0 + s;
            const int a = (int)(cp[j] - nz0), b = (int)(cp[j + 1] - nz0);
            AccT acc = 0;
            for (int e = a; e < b; ++e) acc += buf[e];
            epi.column(j, acc);
        }
        __syncthreads();
        return;
    }
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
            if (s < nseg && lane == 0) buf[s] = acc;
        }
        __syncthreads();
        for (int s = threadIdx.x; s < nseg; s += kBlock) epi.column(tl.seg0 + s, buf[s]);
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
    __shared__ double buf[kTileNnz];
    __shared__ double red[kBlock / 32];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        col_tile<VT, double, Epi>(tl, cp, row, val, v, slots, lcount, splits, epi, buf, red);
    }
}


// ---------------------------------------------------------------------------
// shifted CG (Algorithm 3) kernels; FT = vector type (float or double)
// ---------------------------------------------------------------------------
// Vectors live in the workspace with leading dimension ldw (D rounded up to
// 8, padding kept at zero): r[2][ldw] (r_k in r[k & 1]), p[ldw] (p_{k-1}),
// s[ldw] (X^T v), and the shift state W[S][ldw], P[S][ldw].

template <class FT>
struct Vec16;
template <>
struct Vec16<float> {
    using T = float4;
    static constexpr int n = 4;
    static __device__ __forceinline__ float get(const T &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
    static __device__ __forceinline__ void set(T &v, int i, float x) {
        if (i == 0) v.x = x; else if (i == 1) v.y = x; else if (i == 2) v.z = x; else v.w = x;
    }
};
template <>
struct Vec16<double> {
    using T = double2;
    static constexpr int n = 2;
    static __device__ __forceinline__ double get(const T &v, int i) { return i == 0 ? v.x : v.y; }
    static __device__ __forceinline__ void set(T &v, int i, double x) {
        if (i == 0) v.x = x; else v.y = x;
    }
};

// r_0 = b, p_{-1} = 0, W = 0, P_{-1} = 0; <r,r>, <mu,r>; scalar start values.
template <class FT>
__global__ void __launch_bounds__(kBlock) k_cg_init(int64_t d, int64_t ldw, const double *__restrict__ b, FT *r,
                                                    FT *p, FT *W, FT *P, SolveState *st, double *partials,
                                                    unsigned *counter) {
    __shared__ double red[kBlock / 32];
    const int ns = st->n_shifts;
    const double *mu = st->mu;
    double d0 = 0.0, d1 = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x; j < ldw; j += (int64_t)gridDim.x * kBlock) {
        const FT rj = j < d ? (FT)b[j] : (FT)0;
        r[j] = rj;
        r[ldw + j] = (FT)0;
        p[j] = (FT)0;
        for (int s = 0; s < ns; ++s) {
            W[(int64_t)s * ldw + j] = (FT)0;
            P[(int64_t)s * ldw + j] = (FT)0;
        }
        if (j < d) {
            d0 += (double)rj * (double)rj;
            d1 += mu[j] * (double)rj;
        }
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
        h.active = zero_rhs ? 0 : 1;
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

// phase 1: ut = X p_k - c_k with p_k = r_k + alpha_k p_{k-1}; the first `head`
// entries of p_k (the most frequent features) are formed once per block in
// shared memory, the rest on the fly at the gather.
template <class VT, class FT, int G>
__global__ void __launch_bounds__(kBlock) k_cg_phase1(int64_t n, int head, const int64_t *__restrict__ rp,
                                                      const int32_t *__restrict__ col,
                                                      const VT *__restrict__ val, const FT *__restrict__ r,
                                                      int64_t ldw, const FT *__restrict__ p, FT *__restrict__ ut,
                                                      const SolveState *__restrict__ st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FT *sp = reinterpret_cast<FT *>(smem_raw);
    if (st->done) return;
    const FT a = (FT)st->alpha;
    const double c = st->c;
    const FT *__restrict__ rc = r + (st->k & 1) * ldw;
    for (int f = threadIdx.x; f < head; f += kBlock) sp[f] = form_p<FT>(rc[f], p[f], a);
    __syncthreads();
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
                const FT pj = j < head ? sp[j] : form_p<FT>(rc[j], p[j], a);
                acc += (FT)Val<VT>::get(val, e) * pj;
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
        FT ui = 0, di = 0;
        int8_t yi = 0;
        if (i < n) {
            if (lane == 0) {   // loads of the row's own entries, issued before the gathers
                ui = ut[i];
                di = deg[i];
                yi = y[i];
            }
            const int64_t e1 = rp[i + 1];
            for (int64_t e = rp[i] + lane; e < e1; e += G) acc += sv[e] * ut[col[e]];
        }
#pragma unroll
        for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < n && lane == 0) {
            const double u = (double)ui;
            const double vi = omega * (yi != 0 ? u : 0.0) + al * ((double)di * u - (double)acc);
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

template <class FT>
struct EpiStoreFT {
    FT *s;
    template <class AccT>
    __device__ __forceinline__ void column(int64_t j, AccT x) { s[j] = (FT)x; }
    template <class AccT>
    __device__ __forceinline__ void column_block(int64_t j, AccT x) {
        if (threadIdx.x == 0) s[j] = (FT)x;
    }
};

// phase 3a: s = X^T v (column tiles)
template <class VT, class FT>
__global__ void __launch_bounds__(kBlock) k_cg_phase3a(const Tile *__restrict__ tiles, int ntiles,
                                                       const int64_t *__restrict__ cp,
                                                       const int32_t *__restrict__ row, const VT *__restrict__ val,
                                                       const FT *__restrict__ v, FT *__restrict__ s,
                                                       const SolveState *__restrict__ st, FT *slots,
                                                       unsigned *lcount, const SplitSeg *__restrict__ splits) {
    __shared__ FT buf[kTileNnz];
    __shared__ FT redf[kBlock / 32];
    if (st->done) return;
    EpiStoreFT<FT> epi{s};
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        col_tile<VT, FT, EpiStoreFT<FT>>(tl, cp, row, val, v, slots, lcount, splits, epi, buf, redf);
    }
}

// block-cached scalars of phase 3b
template <class FT>
struct P3Shared {
    double alpha, gamma, t, sigma0;
    int nact;
    int act[kMaxShifts];
    FT zk[kMaxShifts], ak[kMaxShifts], gk[kMaxShifts];
};

// phase 3b: q = s - mu t + sigma0 p_k;  r_{k+1} = r_k + gamma_k q;  p <- p_k;
// P^s_k = zeta^s_k r_k + alpha^s_k P^s_{k-1};  W^s_{k+1} = W^s_k - gamma^s_k P^s_k
// over the flattened (1 + active shifts) x columns space, 16-byte vectors for
// the shift state; then alpha_{k+1}, <mu, p_{k+1}>, <p_{k+1}, p_{k+1}>, stop tests.
template <class FT>
__global__ void __launch_bounds__(kBlock) k_cg_phase3b(int64_t d, int64_t ldw, const FT *__restrict__ s,
                                                       FT *__restrict__ r, FT *__restrict__ p, FT *__restrict__ W,
                                                       FT *__restrict__ P, SolveState *st, double *partials,
                                                       unsigned *counter) {
    using V = typename Vec16<FT>::T;
    constexpr int VW = Vec16<FT>::n;
    __shared__ double red[kBlock / 32];
    __shared__ P3Shared<FT> sm;
    if (st->done) return;
    if (threadIdx.x == 0) {
        sm.alpha = st->alpha;
        sm.gamma = st->gamma;
        sm.t = st->t;
        sm.sigma0 = st->sigma0;
        int na = 0;
        for (int q = 0; q < st->n_shifts; ++q) {
            const ShiftState &h = st->sh[q];
            if (!h.active) continue;
            sm.act[na] = q;
            sm.zk[na] = (FT)h.z;
            sm.ak[na] = (FT)h.a;
            sm.gk[na] = (FT)h.g;
            ++na;
        }
        sm.nact = na;
    }
    __syncthreads();
    const int par = st->k & 1;
    const FT *__restrict__ rc = r + par * ldw;
    FT *__restrict__ rn = r + (par ^ 1) * ldw;
    const double *__restrict__ mu = st->mu;
    const FT al = (FT)sm.alpha;
    const uint32_t nch = (uint32_t)(ldw / VW);
    const uint32_t total = (uint32_t)(sm.nact + 1) * nch;
    double d0 = 0.0, d1 = 0.0, d2 = 0.0;
    for (uint32_t idx = blockIdx.x * kBlock + threadIdx.x; idx < total; idx += gridDim.x * kBlock) {
        const uint32_t a = idx / nch;
        const int64_t j0 = (int64_t)(idx - a * nch) * VW;
        if (a == 0) {
#pragma unroll
            for (int u = 0; u < VW; ++u) {
                const int64_t j = j0 + u;
                if (j >= d) break;
                const FT rj = rc[j];
                const FT pk = form_p<FT>(rj, p[j], al);
                const double mj = mu[j];
                const double q = (double)s[j] - mj * sm.t + sm.sigma0 * (double)pk;
                const FT rnj = (FT)((double)rj + sm.gamma * q);
                rn[j] = rnj;
                p[j] = pk;
                d0 += (double)rnj * (double)rnj;
                d1 += mj * (double)rnj;
                d2 += (double)rnj * (double)pk;
            }
        } else {
            const int q = sm.act[a - 1];
            const FT z = sm.zk[a - 1], aa = sm.ak[a - 1], g = sm.gk[a - 1];
            const V rv = *reinterpret_cast<const V *>(rc + j0);
            V pv = *reinterpret_cast<const V *>(P + (int64_t)q * ldw + j0);
            V wv = *reinterpret_cast<const V *>(W + (int64_t)q * ldw + j0);
#pragma unroll
            for (int u = 0; u < VW; ++u) {
                const FT pn = z * Vec16<FT>::get(rv, u) + aa * Vec16<FT>::get(pv, u);
                Vec16<FT>::set(pv, u, pn);
                Vec16<FT>::set(wv, u, Vec16<FT>::get(wv, u) - g * pn);
            }
            *reinterpret_cast<V *>(P + (int64_t)q * ldw + j0) = pv;
            *reinterpret_cast<V *>(W + (int64_t)q * ldw + j0) = wv;
        }
    }
    double mine[3];
    mine[0] = block_sum(d0, red);
    mine[1] = block_sum(d1, red);
    mine[2] = block_sum(d2, red);
    if (!arrive_last<3>(mine, partials, counter)) return;
    double tot[3];
    reduce_partials<3>(partials, gridDim.x, tot, red);
    __shared__ double s_alpha_new, s_rnorm;
    if (threadIdx.x == 0) {
        const double rr_new = tot[0];
        const double an = rr_new / st->rr;
        const double c_new = tot[1] + an * st->c;
        const double pp_new = rr_new + 2.0 * an * tot[2] + an * an * st->pp;
        if (!isfinite(rr_new) || !isfinite(an)) st->status = SDA_ERR_BREAKDOWN;
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
    for (int q = threadIdx.x; q < st->n_shifts; q += kBlock) {
        ShiftState &h = st->sh[q];
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
        for (int q = 0; q < st->n_shifts; ++q) na += st->sh[q].active;
        st->nactive = na;
        st->done = (na == 0 || k >= st->limit || st->status != SDA_OK) ? 1 : 0;
    }
}

}  // namespace sda
