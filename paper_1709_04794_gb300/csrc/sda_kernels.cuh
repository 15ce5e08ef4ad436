// Device kernels of the operator apply and of the shifted-CG iteration.
//
// One iteration of Algorithm 3 on the centred operator
//   (B + sigma0 I) p = (X - 1 mu^T)^T M (X - 1 mu^T) p + sigma0 p,
//   M = omega P_l + alpha L,  L = D - S                        (eq. 7, Alg. 7, Sec. 3.2.3)
// runs as four kernels:
//   phase 1  (rows of X, k_rowhead):  ut = X p_k - <mu, p_k> 1   (p_k = r_k + alpha_k p_{k-1};
//                             its frequent head formed once per block in shared memory)
//   phase 2  (rows of S, k_rowpass<EpiP2>):  v = omega P_l ut + alpha (D ut - S ut);
//                             block parts of <ut, v> and 1^T v
//   phase 3a (columns of X, k_colblk):  s_r = X_r^T v for each range r of rows; its stream
//                             warps close phase 2 (gamma_k, zeta^s_{k+1} / zeta^s_k, gamma^s_k)
//                             and update P^s_k = zeta^s_k r_k + alpha^s_k P^s_{k-1},
//                             W^s_{k+1} = W^s_k - gamma^s_k P^s_k for the active shifts
//   phase 3b (stream over D, k_cg_phase3b):  s = sum_r s_r;  q = s - mu (1^T v) + sigma0 p_k;
//                             r_{k+1} = r_k + gamma_k q;  <r,r>, <mu,r>, <r,p_k>
//                             -> alpha_{k+1}, <mu,p_{k+1}>, <p_{k+1},p_{k+1}>, stop tests
// <p, (B + sigma0) p> = <ut, v> + sigma0 <p, p> is known after phase 2, so q is
// never stored; <mu, p> and <p, p> follow from recurrences on the phase-3b dots.
// The scalar work of phase 3b runs in the block that finishes last, that of
// phase 2 in every block of phase 3a from phase 2's block parts (no block ever
// waits for another).
//
// k_rowpass (G lanes per row, unrolled independent loads, register sums) serves
// the rows of S and the FP64 operator pieces; k_colpass (column tiles over the
// whole CSC, gathers from global memory) the FP64 operator pieces; k_segpass
// (shared-memory staged tiles) the allocation-free operator apply.
#pragma once

#include "sda_operator.cuh"

namespace sda {

template <class FT>
__device__ __forceinline__ FT form_p(FT r, FT p, FT a);
template <>
__device__ __forceinline__ float form_p<float>(float r, float p, float a) { return fmaf(a, p, r); }
template <>
__device__ __forceinline__ double form_p<double>(double r, double p, double a) { return fma(a, p, r); }

// interleaved {r, p} pair of the CG vectors
template <class FT>
struct RPair;
template <>
struct RPair<float> {
    using T = float2;
};
template <>
struct RPair<double> {
    using T = double2;
};

// ---------------------------------------------------------------------------
// segmented sums over one tile
// ---------------------------------------------------------------------------
template <class AccT>
struct TileSmem {
    AccT buf[kTileNnz];       // products of the tile
    AccT sums[kTileSegs];     // segment sums
    int offs[kTileSegs + 1];  // segment starts relative to the tile
    AccT red[kBlock / 32];
    int last;
};

// Epi must provide
//   tile(i0, nseg, sums)   the whole block, the sums of segments i0 .. i0 + nseg - 1 (shared)
//   segment_block(i, sum)  the whole block, one segment (sum valid in every thread)
// EpiPerSegment supplies tile() for epilogues with a per-segment segment(i, sum).
template <class VT, class AccT, class Gather, class Epi>
__device__ __forceinline__ void seg_tile(const Tile &tl, const int64_t *__restrict__ ptr,
                                         const int32_t *__restrict__ idx, const VT *__restrict__ val,
                                         const Gather &gather, Epi &epi, TileSmem<AccT> &sh, AccT *slots,
                                         unsigned *lcount, const SplitSeg *__restrict__ splits) {
    if (tl.lanes > 0) {
        const int64_t nz0 = tl.nz0;
        const int nnz = (int)(tl.nz1 - nz0);
        const int nseg = tl.seg1 - tl.seg0;
        for (int s = threadIdx.x; s <= nseg; s += kBlock) sh.offs[s] = (int)(ptr[tl.seg0 + s] - nz0);
#pragma unroll 4
        for (int e = threadIdx.x; e < nnz; e += kBlock)
            sh.buf[e] = (AccT)Val<VT>::get_cs(val, nz0 + e) * gather(__ldcs(idx + nz0 + e));
        __syncthreads();
        const int G = tl.lanes;
        if (G == 1) {
            for (int s = threadIdx.x; s < nseg; s += kBlock) {
                AccT acc = 0;
                for (int e = sh.offs[s]; e < sh.offs[s + 1]; ++e) acc += sh.buf[e];
                sh.sums[s] = acc;
            }
        } else {
            const int ngroups = kBlock / G, g = threadIdx.x / G, lane = threadIdx.x % G;
            for (int base = 0; base < nseg; base += ngroups) {
                const int s = base + g;
                AccT acc = 0;
                if (s < nseg)
                    for (int e = sh.offs[s] + lane; e < sh.offs[s + 1]; e += G) acc += sh.buf[e];
                for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (s < nseg && lane == 0) sh.sums[s] = acc;
            }
        }
        __syncthreads();
        epi.tile(tl.seg0, nseg, sh.sums);
        __syncthreads();
        return;
    }
    AccT acc = 0;
#pragma unroll 4
    for (int64_t e = tl.nz0 + threadIdx.x; e < tl.nz1; e += kBlock)
        acc += (AccT)Val<VT>::get_cs(val, e) * gather(__ldcs(idx + e));
    acc = block_sum(acc, sh.red);
    if (tl.slot < 0) {
        epi.segment_block(tl.seg0, acc);
        return;
    }
    // one chunk of a split segment: the chunk that arrives last adds the chunks in order
    if (threadIdx.x == 0) {
        slots[tl.slot] = acc;
        sh.last = (arrive(&lcount[tl.lseg]) == (unsigned)splits[tl.lseg].nchunks - 1u);
    }
    __syncthreads();
    if (sh.last) {
        const SplitSeg sp = splits[tl.lseg];
        AccT tot = 0;
        for (int c = 0; c < sp.nchunks; ++c) tot += __ldcg(slots + sp.slot0 + c);
        if (threadIdx.x == 0) lcount[tl.lseg] = 0u;
        epi.segment_block(tl.seg0, tot);
    }
    __syncthreads();
}

// Epi additionally provides skip() (run finished), begin() and end() (block
// dots and the last block's scalar work).  Gather provides begin() and
// operator()(column) -> AccT.
template <class VT, class AccT, class Gather, class Epi>
__global__ void __launch_bounds__(kBlock) k_segpass(const Tile *__restrict__ tiles, int ntiles,
                                                    const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                                    const VT *__restrict__ val, Gather gather, Epi epi, AccT *slots,
                                                    unsigned *lcount, const SplitSeg *__restrict__ splits) {
    __shared__ TileSmem<AccT> sh;
    __shared__ typename Epi::Shared esh;
    if (epi.skip()) return;
    gather.begin();
    epi.begin(esh);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        seg_tile<VT, AccT, Gather, Epi>(tl, ptr, idx, val, gather, epi, sh, slots, lcount, splits);
    }
    epi.end(esh);
}

struct EpiNoPre {
    struct Pre {};
};

// Row pass for segments of similar, moderate length (rows of X, rows of S):
// G lanes per row, each lane loads up to U (index, value) pairs of its row at
// once (predicated, evict-first) and then issues their U gathers together; the
// row sum is an xor tree over the G lanes; no shared memory.  Rows longer than
// G * U take several rounds.  Epi::segment(i, sum) runs on the row's first lane.
template <class E, class = void>
struct EpiHasPre : std::false_type {};
template <class E>
struct EpiHasPre<E, std::void_t<typename E::Pre>> : std::true_type {};

template <class VT, class AccT, int G, int U, class Gather, class Epi>
__global__ void __launch_bounds__(kBlock) k_rowpass(int64_t n, const int64_t *__restrict__ rp,
                                                    const int32_t *__restrict__ idx, const VT *__restrict__ val,
                                                    Gather gather, Epi epi) {
    __shared__ typename Epi::Shared esh;
    if (epi.skip()) return;
    gather.begin();
    epi.begin(esh);
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x % G;
    const int64_t warp = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kBlock) >> 5;
    // the row pointers of a warp's next round load during the current one
    int64_t p0 = 0, p1 = 0;
    {
        const int64_t i = warp * RPW + (threadIdx.x & 31) / G;
        if (i < n) {
            p0 = rp[i];
            p1 = rp[i + 1];
        }
    }
    for (int64_t base = warp * RPW; base < n; base += nwarps * RPW) {
        const int64_t i = base + (threadIdx.x & 31) / G;
        const int64_t e0 = p0;
        const int len = (int)(p1 - p0);
        {
            const int64_t in = i + nwarps * RPW;
            if (in < n) {
                p0 = rp[in];
                p1 = rp[in + 1];
            }
        }
        // an epilogue with a Pre type reads its per-row inputs before the row sum
        typename std::conditional<EpiHasPre<Epi>::value, Epi, EpiNoPre>::type::Pre pre{};
        if constexpr (EpiHasPre<Epi>::value)
            if (i < n && lane == 0) pre = epi.pre(i);
        AccT acc = 0;
        if (i < n) {
            const int32_t *__restrict__ ip = idx + e0;
            const VT *__restrict__ vp = val + (val ? e0 : 0);
            for (int eb = lane; eb < len; eb += G * U) {
                int32_t jj[U];
                AccT vv[U], gg[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = eb + u * G;
                    const bool ok = e < len;
                    jj[u] = ok ? __ldcs(ip + e) : -1;
                    vv[u] = ok ? (AccT)Val<VT>::get_cs(vp, e) : (AccT)0;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) gg[u] = jj[u] >= 0 ? gather(jj[u]) : (AccT)0;
#pragma unroll
                for (int u = 0; u < U; ++u) acc += vv[u] * gg[u];
            }
        }
#pragma unroll
        for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < n && lane == 0) {
            if constexpr (EpiHasPre<Epi>::value)
                epi.segment(i, acc, pre);
            else
                epi.segment(i, acc);
        }
    }
    epi.end(esh);
}

// ---------------------------------------------------------------------------
// gathers
// ---------------------------------------------------------------------------
template <class AccT, class T>
struct GatherVec {
    const T *__restrict__ v;
    __device__ __forceinline__ void begin() {}
    __device__ __forceinline__ AccT operator()(int32_t j) const { return (AccT)v[j]; }
};

// ---------------------------------------------------------------------------
// epilogues
// ---------------------------------------------------------------------------
struct NoShared {};

// one thread per segment, consecutive segments on consecutive threads
#define SDA_TILE_PER_SEGMENT                                                        \
    template <class AccT>                                                           \
    __device__ __forceinline__ void tile(int64_t i0, int nseg, const AccT *sums) {  \
        for (int s = threadIdx.x; s < nseg; s += kBlock) segment(i0 + s, sums[s]);  \
    }

// out_i = sum - (csub ? *csub : 0)
template <class OT>
struct EpiStore {
    using Shared = NoShared;
    OT *out;
    const double *csub;
    const SolveState *st;   // optional: skip when the run is finished
    double c;
    SDA_TILE_PER_SEGMENT
    __device__ __forceinline__ bool skip() const { return st && st->done; }
    __device__ __forceinline__ void begin(Shared &) { c = csub ? *csub : 0.0; }
    template <class AccT>
    __device__ __forceinline__ void segment(int64_t i, AccT s) {
        out[i] = csub ? (OT)((double)s - c) : (OT)s;
    }
    template <class AccT>
    __device__ __forceinline__ void segment_block(int64_t i, AccT s) {
        if (threadIdx.x == 0) segment(i, s);
    }
    __device__ __forceinline__ void end(Shared &) {}
};

// FP64 Laplacian rows of the operator apply: v_i = omega [y_i != 0] u_i + alpha (D_ii u_i - s_i)
struct EpiLap64 {
    using Shared = NoShared;
    double *v;
    const double *u, *deg;
    const int8_t *y;
    double omega, alpha;
    SDA_TILE_PER_SEGMENT
    __device__ __forceinline__ bool skip() const { return false; }
    __device__ __forceinline__ void begin(Shared &) {}
    __device__ __forceinline__ void segment(int64_t i, double s) {
        const double ui = u[i];
        v[i] = omega * (y[i] != 0 ? ui : 0.0) + alpha * (deg[i] * ui - s);
    }
    __device__ __forceinline__ void segment_block(int64_t i, double s) {
        if (threadIdx.x == 0) segment(i, s);
    }
    __device__ __forceinline__ void end(Shared &) {}
};

// FP64 columns of the operator apply: q_j = s_j - mu_j t + sigma p_j
struct EpiApply {
    using Shared = NoShared;
    double *q;
    const double *mu, *p, *t;
    double sigma, tv;
    SDA_TILE_PER_SEGMENT
    __device__ __forceinline__ bool skip() const { return false; }
    __device__ __forceinline__ void begin(Shared &) { tv = *t; }
    __device__ __forceinline__ void segment(int64_t j, double s) { q[j] = s - mu[j] * tv + sigma * p[j]; }
    __device__ __forceinline__ void segment_block(int64_t j, double s) {
        if (threadIdx.x == 0) segment(j, s);
    }
    __device__ __forceinline__ void end(Shared &) {}
};

// phase 2: v_i = omega [y_i != 0] ut_i + alpha (D_ii ut_i - s_i); dots <ut, v>, 1^T v;
// the last block forms gamma_k, then zeta^s_{k+1} / zeta^s_k and gamma^s_k of every
// active shift, and writes the compact stream parameters.  Per-row arithmetic
// and the per-thread dots are in the vector type (D_ii ut_i - s_i with one
// rounding); the block and grid sums in FP64.
template <class FT>
struct EpiP2 {
    struct Shared {
        double red[kRedDoubles];
    };
    using Part = typename CompSum<FT>::Part;
    FT *v;
    const FT *ut, *deg;
    SolveState *st;
    double *partials;
    const int8_t *y;
    FT omega, al;
    CompSum<FT> d[2];   // <ut, v>, 1^T v (compensated: 1^T v vanishes in exact arithmetic)
    SDA_TILE_PER_SEGMENT
    __device__ __forceinline__ bool skip() const { return st->done != 0; }
    __device__ __forceinline__ void begin(Shared &) {
        y = st->labels;
        omega = (FT)st->omega;
        al = (FT)st->alpha_l;
    }
    // the row's own inputs, read before its sum
    struct Pre {
        FT u, dg;
        int y;
    };
    __device__ __forceinline__ Pre pre(int64_t i) const { return Pre{ut[i], deg[i], (int)y[i]}; }
    __device__ __forceinline__ void segment(int64_t i, FT s, const Pre &pr) {
        const FT u = pr.u;
        const FT lap = fma(pr.dg, u, -s);
        const FT vf = fma(al, lap, pr.y != 0 ? omega * u : (FT)0);
        v[i] = vf;
        d[0].add(u * vf);
        d[1].add(vf);
    }
    __device__ __forceinline__ void segment(int64_t i, FT s) { segment(i, s, pre(i)); }
    __device__ __forceinline__ void segment_block(int64_t i, FT s) {
        if (threadIdx.x == 0) segment(i, s);
    }
    // the block's parts go to partials[block]; the scalar step that closes the
    // phase (gamma_k, the shift ratios) runs in the column pass (stream_scalars)
    __device__ void end(Shared &sh) {
        Part mine[2];
        Part *red = reinterpret_cast<Part *>(sh.red);
        block_parts<2, FT>(d, mine, red);
        if (threadIdx.x == 0) {
            Part *parts = reinterpret_cast<Part *>(partials);
            parts[(int64_t)blockIdx.x * 2 + 0] = mine[0];
            parts[(int64_t)blockIdx.x * 2 + 1] = mine[1];
        }
    }
};

// ---------------------------------------------------------------------------
// shifted CG (Algorithm 3): start and vector/shift-state update
// ---------------------------------------------------------------------------
// Workspace vectors have leading dimension ldw (D rounded up to 8, padding kept
// at zero): RP[2][ldw] interleaved {r, p} (RP[k & 1] holds {r_k, p_{k-1}}),
// s[ldw] = X^T v, and the shift state W[S][ldw], P[S][ldw].

template <class FT>
struct Vec16;
template <>
struct Vec16<float> {
    using T = float4;
    static constexpr int n = 4;
};
template <>
struct Vec16<double> {
    using T = double2;
    static constexpr int n = 2;
};
__device__ __forceinline__ float v16_get(const float4 &v, int i) {
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}
__device__ __forceinline__ void v16_set(float4 &v, int i, float x) {
    if (i == 0) v.x = x;
    else if (i == 1) v.y = x;
    else if (i == 2) v.z = x;
    else v.w = x;
}
__device__ __forceinline__ double v16_get(const double2 &v, int i) { return i == 0 ? v.x : v.y; }
__device__ __forceinline__ void v16_set(double2 &v, int i, double x) {
    if (i == 0) v.x = x;
    else v.y = x;
}

// RP[0] = {b, 0}, RP[1] = 0, W = 0, P_{-1} = 0; <r,r>, <mu,r>; scalar start values
template <class FT>
__global__ void __launch_bounds__(kBlock) k_cg_init(int64_t d, int64_t ldw, const double *__restrict__ b,
                                                    typename RPair<FT>::T *rp, FT *W, FT *P, SolveState *st,
                                                    double *partials, unsigned *counter) {
    using R = typename RPair<FT>::T;
    __shared__ double red[kRedDoubles];
    const int ns = st->n_shifts;
    const double *mu = st->mu;
    double dd[2] = {0.0, 0.0};
    for (int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x; j < ldw; j += (int64_t)gridDim.x * kBlock) {
        const FT rj = j < d ? (FT)b[j] : (FT)0;
        R x;
        x.x = rj;
        x.y = (FT)0;
        rp[j] = x;
        x.x = (FT)0;
        rp[ldw + j] = x;
        for (int s = 0; s < ns; ++s) {
            W[(int64_t)s * ldw + j] = (FT)0;
            P[(int64_t)s * ldw + j] = (FT)0;
        }
        if (j < d) {
            dd[0] += (double)rj * (double)rj;
            dd[1] += mu[j] * (double)rj;
        }
    }
    double mine[2];
    block_dots<2>(dd, mine, red);
    if (!arrive_last<2>(mine, partials, counter)) return;
    double tot[2];
    grid_dots<2>(partials, gridDim.x, tot, red);
    if (threadIdx.x == 0) {
        st->rr = tot[0];
        st->bnorm = sqrt(tot[0]);
        st->inv_bnorm = st->bnorm > 0.0 ? 1.0 / st->bnorm : 0.0;
        st->c = tot[1];
        st->pp = tot[0];
        st->alpha = 0.0;
        st->gamma = 0.0;
        st->gamma_prev = 1.0;
        st->t = 0.0;
        st->k = 0;
        // a right-hand side with a non-finite entry stops the run before its
        // first iteration (reported as a breakdown, not as a zero right-hand side)
        st->status = (isfinite(tot[0]) && isfinite(tot[1])) ? SDA_OK : SDA_ERR_BREAKDOWN;
        *counter = 0u;
    }
    __syncthreads();
    const bool zero_rhs = !(st->bnorm > 0.0);
    int act = 0;
    if (threadIdx.x < ns) {
        ShiftState &h = st->sh[threadIdx.x];
        h.z_prev = 1.0;
        h.z = 1.0;
        h.ratio = 1.0;
        h.g = 0.0;
        h.a = 0.0;
        h.res = zero_rhs ? 0.0 : 1.0;
        h.active = zero_rhs ? 0 : 1;
        h.iters = 0;
        act = h.active;
    }
    const int na = __syncthreads_count(act);
    if (threadIdx.x == 0) {
        st->nactive = na;
        st->done = (na == 0 || st->limit <= 0) ? 1 : 0;
    }
}

// Column pass X^T v: long columns (lanes == 0) as whole-block tiles, split
// across blocks when longer than kTileNnz; the other tiles with `lanes` lanes per
// column, each lane loading up to U (row, value) pairs at once and issuing their
// gathers together; xor-tree sum over the lanes; no shared memory.
// Epi::segment(j, sum) runs on the column's first lane, segment_block for
// whole-block columns.
template <class VT, class AccT, int U, class Epi>
__global__ void __launch_bounds__(kBlock) k_colpass(const Tile *__restrict__ tiles, int ntiles,
                                                    const int64_t *__restrict__ cp, const int32_t *__restrict__ row,
                                                    const VT *__restrict__ val, const AccT *__restrict__ v,
                                                    AccT *slots, unsigned *lcount, const SplitSeg *__restrict__ splits,
                                                    Epi epi) {
    __shared__ typename Epi::Shared esh;
    __shared__ AccT red[kBlock / 32];
    __shared__ int last;
    if (epi.skip()) return;
    epi.begin(esh);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        if (tl.lanes > 0) {
            const int G = tl.lanes, ngroups = kBlock / G;
            const int g = threadIdx.x / G, lane = threadIdx.x % G;
            const int nseg = tl.seg1 - tl.seg0;
            for (int base = 0; base < nseg; base += ngroups) {
                const int s = base + g;
                AccT acc = 0;
                if (s < nseg) {
                    const int64_t j = tl.seg0 + s;
                    const int64_t e0 = cp[j];
                    const int len = (int)(cp[j + 1] - e0);
                    const int32_t *rowj = row + e0;
                    const VT *valj = val + (val ? e0 : 0);
                    for (int eb = lane; eb < len; eb += G * U) {
                        int32_t ii[U];
                        AccT vv[U], gg[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            const int e = eb + u * G;
                            const bool ok = e < len;
                            ii[u] = ok ? __ldcs(rowj + e) : -1;
                            vv[u] = ok ? (AccT)Val<VT>::get_cs(valj, e) : (AccT)0;
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u) gg[u] = ii[u] >= 0 ? v[ii[u]] : (AccT)0;
#pragma unroll
                        for (int u = 0; u < U; ++u) acc += vv[u] * gg[u];
                    }
                }
                for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (s < nseg && lane == 0) epi.segment(tl.seg0 + s, acc);
            }
            continue;
        }
        AccT acc = 0;
#pragma unroll 4
        for (int64_t e = tl.nz0 + threadIdx.x; e < tl.nz1; e += kBlock)
            acc += (AccT)Val<VT>::get_cs(val, e) * v[__ldcs(row + e)];
        acc = block_sum(acc, red);
        if (tl.slot < 0) {
            epi.segment_block(tl.seg0, acc);
            continue;
        }
        if (threadIdx.x == 0) {
            slots[tl.slot] = acc;
            last = (arrive(&lcount[tl.lseg]) == (unsigned)splits[tl.lseg].nchunks - 1u);
        }
        __syncthreads();
        if (last) {
            const SplitSeg sp = splits[tl.lseg];
            AccT tot = 0;
            for (int c = 0; c < sp.nchunks; ++c) tot += __ldcg(slots + sp.slot0 + c);
            if (threadIdx.x == 0) lcount[tl.lseg] = 0u;
            epi.segment_block(tl.seg0, tot);
        }
        __syncthreads();
    }
    epi.end(esh);
}

// Row pass ut = X p_k - <mu, p_k> 1 (Sec. 3.2.3, first identity) with the
// frequent head of p_k in shared memory.  Features are numbered by decreasing
// frequency, so p_k[0, head) serves most gathers: every block forms it once
// from the {r_k, p_{k-1}} pairs (p_k = r_k + alpha_k p_{k-1}); the other
// features read their pair from global memory.  Rows come padded with zero
// entries (column 0) to whole quads: one 16-byte load brings four column
// indices.  G lanes per row, two quads per lane in flight (more flood the
// shared-memory pipe with gathers); lane 0 of the row's group writes ut_i.
template <class VT, class FT, int G>
__global__ void __launch_bounds__(kColBlk, kColBlkPerSm) k_rowhead(int64_t n, int head, int64_t ldw,
                                                                  const int64_t *__restrict__ rp,
                                                                  const int32_t *__restrict__ col,
                                                                  const VT *__restrict__ val,
                                                                  const typename RPair<FT>::T *__restrict__ pairs,
                                                                  FT *__restrict__ ut, const SolveState *st) {
    using R = typename RPair<FT>::T;
    extern __shared__ __align__(16) unsigned char rowhead_smem[];
    FT *ps = reinterpret_cast<FT *>(rowhead_smem);
    if (st->done) return;
    const R *__restrict__ a = pairs + (st->k & 1) * ldw;
    const FT al = (FT)st->alpha, c = (FT)st->c;
    if constexpr (std::is_same<FT, float>::value) {
        // two pairs per 16-byte load, four loads per thread in flight
        const float4 *src = reinterpret_cast<const float4 *>(a);
        float2 *dst = reinterpret_cast<float2 *>(ps);
        const int nv = head / 2;
        for (int i0 = threadIdx.x; i0 < nv; i0 += 4 * kColBlk) {
            float4 x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i0 + u * kColBlk < nv) x[u] = src[i0 + u * kColBlk];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i0 + u * kColBlk < nv)
                    dst[i0 + u * kColBlk] = make_float2(fmaf(al, x[u].y, x[u].x), fmaf(al, x[u].w, x[u].z));
        }
    } else {
        for (int i0 = threadIdx.x; i0 < head; i0 += 4 * kColBlk) {
            R x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i0 + u * kColBlk < head) x[u] = a[i0 + u * kColBlk];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i0 + u * kColBlk < head) ps[i0 + u * kColBlk] = form_p<FT>(x[u].x, x[u].y, al);
        }
    }
    __syncthreads();
    const int4 *__restrict__ colq = reinterpret_cast<const int4 *>(col);
    auto gat = [&](int j) -> FT { return j < head ? ps[j] : form_p<FT>(a[j].x, a[j].y, al); };
    auto quad = [&](int64_t q, bool ok) -> FT {
        int4 ci = make_int4(0, 0, 0, 0);
        FT x[4] = {(FT)0, (FT)0, (FT)0, (FT)0};
        if (ok) {
            ci = __ldcs(colq + q);
            Quad<VT, FT>::load(val, q, x);
        }
        return x[0] * gat(ci.x) + x[1] * gat(ci.y) + x[2] * gat(ci.z) + x[3] * gat(ci.w);
    };
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x % G;
    const int64_t warp = ((int64_t)blockIdx.x * kColBlk + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kColBlk) >> 5;
    // the row pointers of a warp's next round load during the current one
    int64_t p0 = 0, p1 = 0;
    {
        const int64_t i = warp * RPW + (threadIdx.x & 31) / G;
        if (i < n) {
            p0 = rp[i];
            p1 = rp[i + 1];
        }
    }
    for (int64_t base = warp * RPW; base < n; base += nwarps * RPW) {
        const int64_t i = base + (threadIdx.x & 31) / G;
        const int64_t q0 = p0 >> 2;
        const int nq = (int)((p1 >> 2) - q0);
        {
            const int64_t in = i + nwarps * RPW;
            if (in < n) {
                p0 = rp[in];
                p1 = rp[in + 1];
            }
        }
        FT acc = 0;
        if (i < n) {
            for (int qb = lane; qb < nq; qb += 2 * G) {
                const FT a0 = quad(q0 + qb, true);
                const FT a1 = quad(q0 + qb + G, qb + G < nq);
                acc += a0 + a1;
            }
        }
#pragma unroll
        for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (i < n && lane == 0) ut[i] = acc - c;
    }
}

// r_k values of four (FP32) or two (FP64) consecutive features from the
// interleaved {r, p} pairs
__device__ __forceinline__ void load_r(const float2 *a, int64_t j0, float (&r)[4]) {
    const float4 u = *reinterpret_cast<const float4 *>(a + j0);
    const float4 w = *reinterpret_cast<const float4 *>(a + j0 + 2);
    r[0] = u.x;
    r[1] = u.z;
    r[2] = w.x;
    r[3] = w.z;
}
__device__ __forceinline__ void load_r(const double2 *a, int64_t j0, double (&r)[2]) {
    r[0] = a[j0].x;
    r[1] = a[j0 + 1].x;
}

// Compact scalars of one iteration's shift-state stream (shared memory): the
// active shifts in order and their zeta^s_k, alpha^s_k, gamma^s_k.
template <class FT>
struct ShiftTab {
    int act[kMaxShifts];
    FT zk[kMaxShifts], ak[kMaxShifts], gk[kMaxShifts];
    int nact;
    typename CompSum<FT>::Part wsum[kColBlkStreamWarps][2];   // per-warp parts of phase 2's sums
    int wcount[kMaxShifts / 32];                               // active shifts per 32
};
static_assert(sizeof(ShiftTab<double>) <= kShiftTabBytes && sizeof(ShiftTab<float>) <= kShiftTabBytes,
              "shift table outgrows its shared-memory slot");

// The scalar step that closes phase 2 (Algorithm 3): from the phase's block
// parts of <ut, v> and 1^T v, <p, (B + sigma0) p> = <ut, v> + sigma0 ||p||^2,
// gamma_k = -<r, r> / <p, (B + sigma0) p>, and per active shift
//   zeta_{k+1} / zeta_k = zeta_{k-1} gamma_{k-1} / (gamma_k alpha_k (zeta_{k-1} - zeta_k)
//                          + zeta_{k-1} gamma_{k-1} (1 - (beta - sigma0) gamma_k)),
//   gamma^s_k = gamma_k zeta_{k+1} / zeta_k.
// Run by the NT = kColBlkStreamWarps * 32 stream threads (index sl) of every
// column-pass block on the same parts in a fixed order, so every block gets
// the same values; it fills `tab` (the active shifts' zeta^s_k, alpha^s_k,
// gamma^s_k in shift order) and, in the writer block, the solve state.
// Returns false on breakdown (<p, (B + sigma0) p> <= 0 or not finite).
template <class FT>
__device__ bool stream_scalars(SolveState *st, const typename CompSum<FT>::Part *__restrict__ parts, int nb,
                               ShiftTab<FT> &tab, int sl, bool writer) {
    constexpr int NT = kColBlkStreamWarps * 32;
    using CS = CompSum<FT>;
    const int w = sl >> 5, l = sl & 31;
    // the shift state is read first so that its loads overlap the sum
    const int ns = st->n_shifts;
    ShiftState *h = st->sh + sl;
    int act = 0;
    double zp = 0.0, zk = 0.0, ak = 0.0, dl = 0.0;
    if (sl < ns) {
        act = h->active;
        zp = h->z_prev;
        zk = h->z;
        ak = h->a;
        dl = h->delta;
    }
    const double gp = st->gamma_prev, al_k = st->alpha, rr = st->rr, sigma0 = st->sigma0, pp = st->pp;
    CS a[2];
    for (int b = sl; b < nb; b += NT) {
        CS::add_part(a[0], __ldcg(parts + 2 * (int64_t)b));
        CS::add_part(a[1], __ldcg(parts + 2 * (int64_t)b + 1));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a[0].xor_reduce(o);
        a[1].xor_reduce(o);
    }
    if (l == 0) {
        tab.wsum[w][0] = a[0].part();
        tab.wsum[w][1] = a[1].part();
    }
    asm volatile("bar.sync 1, %0;" ::"r"(NT) : "memory");
    double tot[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        CS t;
#pragma unroll
        for (int q = 0; q < kColBlkStreamWarps; ++q) CS::add_part(t, tab.wsum[q][k]);
        tot[k] = t.to_double();
    }
    const double pq = tot[0] + sigma0 * pp;
    if (!(pq > 0.0) || !isfinite(pq)) {
        if (writer && sl == 0) {
            st->status = SDA_ERR_BREAKDOWN;
            st->done = 1;
        }
        return false;
    }
    const double gam = -rr / pq;
    double gk = 0.0;
    if (act) {
        const double den = gam * al_k * (zp - zk) + zp * gp * (1.0 - dl * gam);
        const double ratio = zp * gp / den;
        gk = gam * ratio;
        if (writer) {
            h->ratio = ratio;
            h->g = gk;
        }
    }
    // compact the active shifts (slot = active shifts before it)
    const unsigned bal = __ballot_sync(0xffffffffu, act);
    if (l == 0 && w < kMaxShifts / 32) tab.wcount[w] = __popc(bal);
    asm volatile("bar.sync 1, %0;" ::"r"(NT) : "memory");
    if (act) {
        int pos = __popc(bal & ((1u << l) - 1u));
        for (int q = 0; q < w; ++q) pos += tab.wcount[q];
        tab.act[pos] = sl;
        tab.zk[pos] = (FT)zk;
        tab.ak[pos] = (FT)ak;
        tab.gk[pos] = (FT)gk;
    }
    if (sl == 0) {
        int na = 0;
        for (int q = 0; q < kMaxShifts / 32; ++q) na += tab.wcount[q];
        tab.nact = na;
        if (writer) {
            st->gamma = gam;
            st->t = tot[1];
            StreamParams &sp = st->sp;
            sp.alpha = al_k;
            sp.gamma = gam;
            sp.t = tot[1];
            sp.sigma0 = sigma0;
            sp.nact = na;
        }
    }
    asm volatile("bar.sync 1, %0;" ::"r"(NT) : "memory");
    return true;
}

// The shift-state stream of iteration k (Algorithm 3, every active shift s):
//   P^s_k = zeta^s_k r_k + alpha^s_k P^s_{k-1};  W^s_{k+1} = W^s_k - gamma^s_k P^s_k
// over items i = q * nch + c (active slot q, 16-byte chunk c), item i to thread
// i mod nthr; (q, c) advance by (nthr / nch, nthr % nch) without a division per
// item, two items per thread in flight.  a: the {r_k, p_{k-1}} pairs.
template <class FT>
__device__ __forceinline__ void shift_stream(int64_t tid, int64_t nthr, int64_t ldw,
                                             const typename RPair<FT>::T *__restrict__ a, FT *__restrict__ W,
                                             FT *__restrict__ P, const ShiftTab<FT> &tab) {
    using V = typename Vec16<FT>::T;
    constexpr int VW = Vec16<FT>::n;
    constexpr int UNROLL = 2;
    const int nch = (int)(ldw / VW), nact = tab.nact;
    int q = (int)(tid / nch), c = (int)(tid - (int64_t)q * nch);
    const int sq = (int)(nthr / nch), sc = (int)(nthr - (int64_t)sq * nch);
    while (q < nact) {
        FT r[UNROLL][VW];
        V pv[UNROLL], wv[UNROLL];
        int64_t off[UNROLL];
        int qq[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            qq[u] = q;
            if (q < nact) {
                const int64_t j0 = (int64_t)c * VW;
                off[u] = (int64_t)tab.act[q] * ldw + j0;
                load_r(a, j0, r[u]);
                pv[u] = *reinterpret_cast<const V *>(P + off[u]);
                wv[u] = *reinterpret_cast<const V *>(W + off[u]);
            }
            q += sq;
            c += sc;
            if (c >= nch) {
                c -= nch;
                ++q;
            }
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            if (qq[u] >= nact) continue;
            const FT z = tab.zk[qq[u]], aa = tab.ak[qq[u]], g = tab.gk[qq[u]];
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                const FT pn = z * r[u][e] + aa * v16_get(pv[u], e);
                v16_set(pv[u], e, pn);
                v16_set(wv[u], e, v16_get(wv[u], e) - g * pn);
            }
            *reinterpret_cast<V *>(P + off[u]) = pv[u];
            *reinterpret_cast<V *>(W + off[u]) = wv[u];
        }
    }
}

// Column pass s = X^T v over ranges of rows (Sec. 3.2.3, second identity, before
// the rank-one term): block b serves range r = b / per_range.  It first copies
// v's slice of rows [r * rb, (r + 1) * rb) into shared memory (cp.async, all
// copies in flight at once); then its warps work the range's warp tiles
// round-robin, with every gather served from that copy.  Entries come in quads
// (segments padded with zero entries to multiples of four): one 8-byte load
// brings four 16-bit local row indices.  A multi-column tile loads all its
// quads and column starts at once, parks the quad sums in the warp's scratch
// and gives each column a group of `lanes` lanes to add them; whole-warp tiles
// take one chunk of a long column, four quads per lane; the chunk of a split
// column that arrives last adds the chunks' parts in a fixed order.  The last
// kColBlkStreamWarps warps of each block run the iteration's shift-state
// stream instead (W, P of the active shifts; none when W is null): they first
// close phase 2 (gamma_k and the shift coefficients, from phase 2's block
// parts, identically in every block; block 0 stores them), then stream, using
// the bandwidth the latency-bound tiles leave.  Sums are
// compensated (CompSum): the frequent features' columns run over most rows and
// cancel (1^T v vanishes), so plain FP32 sums would lose their digits.  The
// sums of range r go to out[r * ldo + j] as CompSum parts; the consumer adds
// the ranges in order.
template <class VT, class AccT>
__global__ void __launch_bounds__(kColBlk, kColBlkPerSm) k_colblk(const Tile *__restrict__ tiles, int per_range,
                                                   int64_t n, int64_t rb, int64_t nseg, int64_t ldo,
                                                   const int64_t *__restrict__ cp, const uint16_t *__restrict__ row,
                                                   const VT *__restrict__ val, const AccT *__restrict__ v,
                                                   typename CompSum<AccT>::Part *__restrict__ out,
                                                   typename CompSum<AccT>::Part *slots,
                                                   unsigned *lcount, const SplitSeg *__restrict__ splits,
                                                   const int32_t *__restrict__ tile_off, SolveState *st,
                                                   int64_t ldw, const typename RPair<AccT>::T *__restrict__ rp,
                                                   AccT *__restrict__ W, AccT *__restrict__ P,
                                                   const typename CompSum<AccT>::Part *__restrict__ p2parts,
                                                   int p2blocks) {
    using CS = CompSum<AccT>;
    extern __shared__ __align__(16) unsigned char colblk_smem[];
    AccT *vs = reinterpret_cast<AccT *>(colblk_smem);
    ShiftTab<AccT> &tab = *reinterpret_cast<ShiftTab<AccT> *>(
        colblk_smem + (rb * (int64_t)sizeof(AccT) + 15) / 16 * 16 + colblk_scratch((int64_t)sizeof(AccT)) -
        kShiftTabBytes);
    if (st && st->done) return;
    const int r = blockIdx.x / per_range, c = blockIdx.x - r * per_range;
    const int64_t r0 = (int64_t)r * rb;
    const int len = (int)min(rb, n - r0);
    // a tile warp's first tile: its descriptor loads now, its quads are
    // prefetched to L2 while the slice of v is staged
    constexpr int TW = kColBlk / 32 - kColBlkStreamWarps;
    const int wib = threadIdx.x >> 5;
    const int t_first = tile_off[r] + c * TW + wib;
    const bool has_first = wib < TW && t_first < tile_off[r + 1];
    Tile first{};
    if (has_first) first = tiles[t_first];
    {
        // v + r0 is 16-byte aligned (rb is a multiple of 256 and v is aligned)
        constexpr int VW = 16 / (int)sizeof(AccT);
        const int n16 = len / VW;
        const char *src = reinterpret_cast<const char *>(v + r0);
        const unsigned dst = (unsigned)__cvta_generic_to_shared(colblk_smem);
        for (int i = threadIdx.x; i < n16; i += kColBlk)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + 16u * (unsigned)i),
                         "l"(src + 16 * (int64_t)i)
                         : "memory");
        for (int i = n16 * VW + threadIdx.x; i < len; i += kColBlk) vs[i] = v[r0 + i];
        if (has_first) {
            // one 128-byte line of the tile's 16-bit indices and of its values per lane and round
            const int64_t e0 = first.nz0, e1 = first.nz1;
            const char *ib = reinterpret_cast<const char *>(row);
            const char *vb = reinterpret_cast<const char *>(val);
            for (int64_t b = (e0 * 2) / 128 + (threadIdx.x & 31); b * 128 < e1 * 2; b += 32)
                asm volatile("prefetch.global.L2 [%0];\n" ::"l"(ib + b * 128));
            for (int64_t b = (e0 * (int64_t)sizeof(VT)) / 128 + (threadIdx.x & 31); b * 128 < e1 * (int64_t)sizeof(VT);
                 b += 32)
                asm volatile("prefetch.global.L2 [%0];\n" ::"l"(vb + b * 128));
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    __syncthreads();
    const uint2 *__restrict__ rowq = reinterpret_cast<const uint2 *>(row);
    const int64_t *__restrict__ cpr = cp + (int64_t)r * (nseg + 1);
    typename CS::Part *__restrict__ outr = out + (int64_t)r * ldo;
    const int lane32 = threadIdx.x & 31;
    // this warp's scratch: quad sums of a multi-column tile, then its column starts
    AccT *qs = reinterpret_cast<AccT *>(colblk_smem + (rb * (int64_t)sizeof(AccT) + 15) / 16 * 16 +
                                        (int64_t)(threadIdx.x >> 5) *
                                            ((int64_t)kWarpTileQuads * (int64_t)sizeof(AccT) + kWarpTilePosBytes));
    int16_t *qpos = reinterpret_cast<int16_t *>(qs + kWarpTileQuads);
    using QL = Quad<VT, AccT>;
    // dot of a quad with the staged slice (four products, rounded sum)
    auto dot4 = [&](uint2 ri, const AccT (&x)[4]) -> AccT {
        return x[0] * vs[ri.x & 0xffffu] + x[1] * vs[ri.x >> 16] + x[2] * vs[ri.y & 0xffffu] + x[3] * vs[ri.y >> 16];
    };
    auto quad = [&](int64_t q, bool ok) -> AccT {
        uint2 ri = make_uint2(0u, 0u);
        AccT x[4] = {(AccT)0, (AccT)0, (AccT)0, (AccT)0};
        if (ok) {
            ri = __ldcs(rowq + q);
            QL::load(val, q, x);
        }
        return dot4(ri, x);
    };
    // one warp tile
    auto work = [&](const Tile &tl) {
        if (tl.lanes > 0) {
            // multi-column tile: at most kWarpTileQuads quads and kWarpTileSegs
            // columns.  All its quads and column starts load at once (coalesced);
            // the quad sums go to the warp's scratch, then `lanes` lanes per
            // column add them (compensated, lane-strided as the quads lie).
            const int64_t q0 = tl.nz0 >> 2;
            const int nq = (int)((tl.nz1 >> 2) - q0);
            const int nsg = tl.seg1 - tl.seg0;
            constexpr int QPL = kWarpTileQuads / 32;
            constexpr int SPL = (kWarpTileSegs + 32) / 32;
            uint2 ri[QPL];
            AccT x[QPL][4];
            int64_t cv[SPL];
#pragma unroll
            for (int u = 0; u < QPL; ++u) {
                const int q = lane32 + 32 * u;
                ri[u] = make_uint2(0u, 0u);
#pragma unroll
                for (int e = 0; e < 4; ++e) x[u][e] = (AccT)0;
                if (q < nq) {
                    ri[u] = __ldcs(rowq + q0 + q);
                    QL::load(val, q0 + q, x[u]);
                }
            }
#pragma unroll
            for (int m = 0; m < SPL; ++m) {
                const int sg = lane32 + 32 * m;
                cv[m] = sg <= nsg ? __ldg(cpr + tl.seg0 + sg) : 0;
            }
#pragma unroll
            for (int m = 0; m < SPL; ++m) {
                const int sg = lane32 + 32 * m;
                if (sg <= nsg) qpos[sg] = (int16_t)((cv[m] >> 2) - q0);
            }
#pragma unroll
            for (int u = 0; u < QPL; ++u) {
                const int q = lane32 + 32 * u;
                if (q < nq) qs[q] = dot4(ri[u], x[u]);
            }
            __syncwarp();
            const int G = tl.lanes, per = 32 / G;
            const int g = lane32 / G, lane = lane32 % G;
            for (int base = 0; base < nsg; base += per) {
                const int sgi = base + g;
                CS acc;
                if (sgi < nsg) {
                    const int e1 = qpos[sgi + 1];
                    for (int e = qpos[sgi] + lane; e < e1; e += G) acc.add(qs[e]);
                }
                for (int o = G >> 1; o > 0; o >>= 1) acc.xor_reduce(o);
                if (sgi < nsg && lane == 0) outr[tl.seg0 + sgi] = acc.part();
            }
            __syncwarp();
            return;
        }
        const int64_t q0 = tl.nz0 >> 2;
        const int nq = (int)((tl.nz1 >> 2) - q0);
        CS acc;
        constexpr int QPL = warp_chunk_nnz((int64_t)sizeof(AccT)) / 128;
        for (int qb = lane32; qb < nq; qb += QPL * 32) {
            AccT a[QPL];
#pragma unroll
            for (int u = 0; u < QPL; ++u) a[u] = quad(q0 + qb + 32 * u, qb + 32 * u < nq);
#pragma unroll
            for (int u = 0; u < QPL; ++u) acc.add(a[u]);
        }
        for (int o = 16; o > 0; o >>= 1) acc.xor_reduce(o);
        if (tl.slot < 0) {
            if (lane32 == 0) outr[tl.seg0] = acc.part();
            return;
        }
        // a chunk of a split column: its part goes to a slot; the warp of the
        // chunk that arrives last adds the column's parts (compensated, fixed
        // shuffle tree)
        int last = 0;
        const SplitSeg sp = splits[tl.lseg];
        if (lane32 == 0) {
            slots[tl.slot] = acc.part();
            last = arrive(&lcount[tl.lseg]) == (unsigned)sp.nchunks - 1u;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
            __syncwarp();
            CS tot;
            for (int q = lane32; q < sp.nchunks; q += 32) CS::add_part(tot, __ldcg(slots + sp.slot0 + q));
            for (int o = 16; o > 0; o >>= 1) tot.xor_reduce(o);
            if (lane32 == 0) {
                lcount[tl.lseg] = 0u;
                outr[tl.seg0] = tot.part();
            }
        }
    };
    // the last kColBlkStreamWarps warps of every block run the shift-state
    // stream of this iteration (bandwidth-bound; the tile warps are bound by
    // latency), the others the range's tiles
    if (wib >= TW) {
        if (W && stream_scalars<AccT>(st, p2parts, p2blocks, tab, threadIdx.x - TW * 32, blockIdx.x == 0))
            shift_stream<AccT>((int64_t)(blockIdx.x * kColBlkStreamWarps + (wib - TW)) * 32 + lane32,
                               (int64_t)gridDim.x * kColBlkStreamWarps * 32, ldw, rp + (st->k & 1) * ldw, W, P, tab);
        return;
    }
    // the range's tiles round-robin over its tile warps (tiles come in column
    // order: long columns first, so every warp gets a mix of long and short
    // ones); the next tile's descriptor loads while a tile is worked
    const int nw = per_range * TW;
    const int t1 = tile_off[r + 1];
    int t = t_first;
    if (has_first) {
        Tile cur = first;
        for (;;) {
            const int tn = t + nw;
            Tile nxt = cur;
            if (tn < t1) nxt = tiles[tn];
            work(cur);
            if (tn >= t1) break;
            cur = nxt;
            t = tn;
        }
    }
}

// phase 3b (stream over D), s_j = sum of the row-range partials of X^T v,
// q_j = s_j - mu_j t + sigma0 p_k,j for every feature:
//   r_{k+1} = r_k + gamma_k q;  RP[k+1] = {r_{k+1}, p_k}
// one grid-stride pass (the shift state of the iteration is streamed by the
// column pass, which runs before).  The scalars arrive in the compact block
// st->sp written by phase 2.  Dots <r_{k+1}, r_{k+1}>, <mu, r_{k+1}>,
// <r_{k+1}, p_k>; the last block forms alpha_{k+1}, <mu, p_{k+1}>,
// ||p_{k+1}||^2 and the stop tests.
template <class FT>
struct StreamSmem {
    double alpha, gamma, t, sigma0;
    double red[kRedDoubles];
    double alpha_new, rnorm;
    float gh, gl, sh, sl, tf;   // gamma_k, sigma0 as FP32 pairs, t in FP32 (mixed path)
    int exact;                  // r_{k+1} = 0: every shift's solution is exact, the run ends
};


// r_{k+1} = r_k + gamma_k (s - mu t + sigma0 p_k) in FP32 pairs (s given as the
// pair sjh + sjl), rounded once at the end (the same value as an FP64
// evaluation rounded to FP32 up to ties); the mu t term is kept at FP32
// precision since t = 1^T v vanishes in exact arithmetic.
__device__ __forceinline__ float base_step_f32v(float r, float pk, float sjh, float sjl, float mj, float sh,
                                                float sl, float tf, float gh, float gl) {
    float e0, e1, e2, e3;
    const float bh = two_prod(sh, pk, e0);
    const float bl = fmaf(sl, pk, e0);
    const float qh0 = two_sum(sjh, bh, e1);
    const float ql0 = fmaf(-mj, tf, (e1 + bl) + sjl);
    const float qh = qh0 + ql0;
    const float ql = ql0 - (qh - qh0);
    const float ph = two_prod(gh, qh, e2);
    const float s = two_sum(r, ph, e3);
    return s + ((e3 + e2) + fmaf(gh, ql, gl * qh));
}
__device__ __forceinline__ float base_step_f32(float r, float pk, float sjh, float sjl, float mj,
                                               const StreamSmem<float> &sm) {
    return base_step_f32v(r, pk, sjh, sjl, mj, sm.sh, sm.sl, sm.tf, sm.gh, sm.gl);
}


template <class FT>
__global__ void __launch_bounds__(kBlock) k_cg_phase3b(int64_t d, int64_t ldw,
                                                       const typename CompSum<FT>::Part *__restrict__ s, int nparts,
                                                       typename RPair<FT>::T *__restrict__ rp,
                                                       FT *__restrict__ W, FT *__restrict__ P, SolveState *st,
                                                       double *partials, unsigned *counter) {
    using R = typename RPair<FT>::T;
    __shared__ StreamSmem<FT> sm;
    if (st->done) return;
    {
        const StreamParams &sp = st->sp;
        if (threadIdx.x == 0) {
            sm.alpha = sp.alpha;
            sm.gamma = sp.gamma;
            sm.t = sp.t;
            sm.sigma0 = sp.sigma0;
        }
        if (threadIdx.x == 32) {
            split_f32(sp.gamma, sm.gh, sm.gl);
            split_f32(sp.sigma0, sm.sh, sm.sl);
            sm.tf = (float)sp.t;
        }
    }
    constexpr bool kF32 = std::is_same<FT, float>::value;
    __syncthreads();
    const int par = st->k & 1;
    const R *__restrict__ a = rp + par * ldw;
    R *__restrict__ an_ = rp + (par ^ 1) * ldw;
    // the base recurrence r_{k+1} = r_k + gamma_k q is rounded once to the vector
    // type: FP64 arithmetic on the FP64 path, FP32 pairs on the mixed path (D
    // elements per iteration); the dots are summed in the vector type per warp
    const FT al = (FT)sm.alpha;
    const int64_t tid = (int64_t)blockIdx.x * kBlock + threadIdx.x, nthr = (int64_t)gridDim.x * kBlock;
    CompSum<FT> dd[3];   // compensated: <mu, r> and <r, p> may cancel
    if constexpr (kF32) {
        const float *__restrict__ mu = st->mu32;
        for (int64_t j = tid; j < d; j += nthr) {
            const R x = a[j];
            const float pk = form_p<float>(x.x, x.y, al);
            const float mj = mu[j];
            CompSum<float> sj;
            for (int q = 0; q < nparts; ++q) CompSum<float>::add_part(sj, s[(int64_t)q * ldw + j]);
            const float rnj = base_step_f32(x.x, pk, sj.h, sj.l, mj, sm);
            R y;
            y.x = rnj;
            y.y = pk;
            an_[j] = y;
            dd[0].add(rnj * rnj);
            dd[1].add(mj * rnj);
            dd[2].add(rnj * pk);
        }
    } else {
        const double *__restrict__ mu = st->mu;
        const double t = sm.t, sigma0 = sm.sigma0, gam = sm.gamma;
        for (int64_t j = tid; j < d; j += nthr) {
            const R x = a[j];
            const FT pk = form_p<FT>(x.x, x.y, al);
            const double mj = mu[j];
            CompSum<FT> sj;
            for (int q = 0; q < nparts; ++q) CompSum<FT>::add_part(sj, s[(int64_t)q * ldw + j]);
            const double qj = (double)sj.value() - mj * t + sigma0 * (double)pk;
            const FT rnj = (FT)((double)x.x + gam * qj);
            R y;
            y.x = rnj;
            y.y = pk;
            an_[j] = y;
            dd[0].add(rnj * rnj);
            dd[1].add((FT)mj * rnj);
            dd[2].add(rnj * pk);
        }
    }
    using Part = typename CompSum<FT>::Part;
    Part mine[3];
    Part *red = reinterpret_cast<Part *>(sm.red);
    Part *parts = reinterpret_cast<Part *>(partials);
    block_parts<3, FT>(dd, mine, red);
    if (!arrive_last_parts<3>(mine, parts, counter)) return;
    // the shift state is read before the grid sum so that its loads overlap it
    const int ns = st->n_shifts, sh_q = threadIdx.x;
    ShiftState *h = st->sh + sh_q;
    int act = 0;
    double zk = 0.0, ratio = 0.0;
    if (sh_q < ns) {
        act = h->active;
        zk = h->z;
        ratio = h->ratio;
    }
    const int k = st->k + 1;
    const double tolb = st->tol * st->bnorm, inv_b = st->inv_bnorm;
    const int fixed = st->fixed;
    double tot[3];
    grid_parts<3, FT>(parts, gridDim.x, tot, red);
    if (threadIdx.x == 0) {
        const double rr_new = tot[0];
        const double anw = rr_new / st->rr;
        const double c_new = tot[1] + anw * st->c;
        const double pp_new = rr_new + 2.0 * anw * tot[2] + anw * anw * st->pp;
        if (!isfinite(rr_new) || !isfinite(anw)) st->status = SDA_ERR_BREAKDOWN;
        st->gamma_prev = st->gamma;
        st->alpha = anw;
        st->c = c_new;
        st->pp = pp_new;
        st->rr = rr_new;
        st->k = k;
        sm.alpha_new = anw;
        sm.rnorm = sqrt(rr_new);
        // an exactly vanished residual ends the run (a fixed-iteration run would
        // otherwise go on with p = 0 and divide by <p, (B + sigma0) p> = 0)
        sm.exact = rr_new == 0.0;
        *counter = 0u;
    }
    __syncthreads();
    if (act) {
        const double zn = zk * ratio;
        h->a = sm.alpha_new * ratio * ratio;
        h->z_prev = zk;
        h->z = zn;
        h->iters = k;
        const double rz = fabs(zn) * sm.rnorm;
        h->res = rz * inv_b;
        if (!fixed && (rz < tolb || !(fabs(zn) > 0.0))) act = 0;
        h->active = act;
    }
    const int na = __syncthreads_count(act);
    if (threadIdx.x == 0) {
        st->nactive = na;
        st->done = (na == 0 || k >= st->limit || st->status != SDA_OK || sm.exact) ? 1 : 0;
    }
}

// <a, b> (or the sum of a when b is NULL) into *out, fixed-order reduction
__global__ void __launch_bounds__(kBlock) k_dot_f64(int64_t n, const double *__restrict__ a,
                                                    const double *__restrict__ b, double *out,
                                                    double *partials, unsigned *counter);

}  // namespace sda
