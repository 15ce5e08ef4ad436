// Batched targets: many binary targets that share X and S are solved together,
// kTB targets per batch, one shifted-CG run (Algorithm 3) per target advanced
// in lockstep.  The operator passes become sparse-matrix x dense-block products:
// every vector is stored target-contiguous ([index][kTB]), a group of kTB lanes
// (one lane per target) serves one row or column, the index and value of a
// nonzero are loaded once for the group and the gather of the kTB targets'
// values is one contiguous access.  Per target: its own labels, mu_l, right-hand
// side, CG scalars and shift states (a SolveState each); the shift list is the
// call's.  X and S are streamed once per batch iteration instead of once per
// target.  A batch's iterations run as one graph launch with a device-side loop
// condition; an autotuner picks the passes' schedule.  The same kernels in FP64
// serve the block utilities (FP64 true residuals, projections, adjoint
// contractions, class sums, 16 vectors per pass), whose X passes run in exact
// fixed point where X's values allow it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "sda_kernels.cuh"

namespace sda {

constexpr int kTB = 16;              // targets per batch
constexpr int kTG = kBlock / kTB;    // lane groups per block

// Bounds of every array the batched kernels index with computed offsets: the
// kernels check each such index and skip an access that falls outside,
// recording the first one in BatchCtl::err (reported to the caller).
struct BatchBounds {
    int64_t n, d, ldw, n8, nnz_x, nnz_s, ntiles, nslots, nsplits, npart;
    int64_t nqx;   // quads of the padded row layout of X
};

// value type of the padded row layout (a pattern X stores FP8 ones there)
template <class VT>
using BVT = std::conditional_t<std::is_same<VT, Pattern>::value, __nv_fp8_e4m3, VT>;

struct BatchCtl {
    int32_t k;        // iterations completed
    int32_t done;     // every target of the batch has stopped
    int32_t status;
    int32_t bodies;           // loop bodies run by the device-driven loop (bounds it on its own)
    unsigned long long err;   // first index check that failed: (site << 40) | index; 0 if none
    BatchBounds bb;
};

__device__ __forceinline__ bool in_bounds(BatchCtl *ctl, long long idx, long long bound, int site) {
    if (idx >= 0 && idx < bound) return true;
    atomicCAS(&ctl->err, 0ull, ((unsigned long long)site << 40) | ((unsigned long long)idx & 0xffffffffffull));
    return false;
}
#define BOK(idx, bound, site) in_bounds(const_cast<BatchCtl *>(ctl), (long long)(idx), (long long)(bound), (site))

// per (shift, target) coefficients of the stream, written by phase 2
template <class FT>
struct BatchCoef {
    FT z, a, g;       // zeta_k, alpha^s_k, gamma^s_k
    int32_t active;
};

// Scalars of one iteration k of a lane's base CG run, kept for the stored-basis
// form: a = -gamma_k (the step), b = alpha_{k+1} = <r_{k+1}, r_{k+1}> / <r_k, r_k>,
// rr = <r_k, r_k> (all FP64).  They define the tridiagonal T of the base system.
struct LzStep {
    double a, b, rr;
};

// Device view of the stored basis: slot k (iteration k's base residual r_k, all
// lanes, [ldw][kTB]) lives at tab[k / per_chunk] + (k % per_chunk) * ldw * kTB;
// NULL tab selects the recurrences.
template <class FT>
struct BasisView {
    FT *const *tab;
    int per_chunk;
    LzStep *lz;      // [k][kTB]
};

struct BatchWs {
    int fp64 = -1;
    int64_t d = 0, n = 0, ldw = 0, n8 = 0;
    int ns = 0;
    DevBuf<char> vec;      // pairs [2][ldw][kTB], s parts [ldw][kTB], ut [n8][kTB], v [n8][kTB], p [ldw][kTB]
    DevBuf<char> shift;    // W [ns][ldw][kTB], P [ns][ldw][kTB]
    DevBuf<double> b, mu64;
    DevBuf<float> mu32;
    DevBuf<int8_t> ylab;
    DevBuf<SolveState> st;
    DevBuf<BatchCtl> ctl;
    DevBuf<char> coef;
    DevBuf<double> part, slots;
    DevBuf<double> hparts;     // head column pass: parts [range][head column][kTB] (one 8-byte part each)
    DevBuf<double> sig, r2;    // per-lane shifts and squared residual norms of the FP64 block utilities
    DevBuf<double> wall;       // FP64 solutions of a batch's (target, shift) pairs [target][shift][D]
    DevBuf<double> rbuf;       // residual vectors of up to kTB pairs [lane][D] (refinement right-hand sides)
    // FP64 workspaces, fixed-point X passes: the scaled vector as planes
    // [kTB / kFxNT][len][kFxNT], the per-lane max |z| (bit patterns) and scale exponents
    DevBuf<int2> fx_planes;
    DevBuf<unsigned long long> fx_amax;
    DevBuf<int> fx_k;
    int grid_fx1 = 0, grid_fx3 = 0, grid_fx_head = 0;
    // stored-basis form: chunks of kBasisChunk slots [ldw][kTB] each, their device
    // pointer table (graphs read it, so new chunks need no recapture), the CG scalars
    // of every iteration and the per-(lane, shift) basis coefficients
    std::vector<std::unique_ptr<DevBuf<char>>> bchunks;
    DevBuf<char> btab;
    int btab_cap = 0;
    DevBuf<LzStep> lz;
    DevBuf<double> coefs;
    int shift_ns = 0;          // shifts the W, P buffers hold (recurrence form)
    DevBuf<unsigned> cnt, lcount;
    SolveState *h_st = nullptr;
    BatchCtl *h_ctl = nullptr;
    int grid = 0;                          // every kernel but the sparse passes of the batched solve
    int grid1 = 0, grid2 = 0, grid3a = 0;  // their own grids (occupancy of each)
    int grid_head = 0;                     // grid of the head column pass
    bool head_ready = false;               // its shared-memory attribute set
    int head_items = 4;                    // head pass: work items per resident block (tuned; 0: no head pass)
    bool tuned = false;                    // the schedule of the sparse passes has been picked
    cudaGraphExec_t loop = nullptr;        // device-driven loop: a WHILE node over loop_iters iterations
    int loop_iters = 0, loop_ns = 0, loop_basis = -1, loop_limit = -1;
    cudaStream_t cap_stream = nullptr;
    ~BatchWs() {
        if (loop) cudaGraphExecDestroy(loop);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (h_st) cudaFreeHost(h_st);
        if (h_ctl) cudaFreeHost(h_ctl);
    }
};

// ---------------------------------------------------------------------------
// per-target reductions (thread x holds target x % kTB)
// ---------------------------------------------------------------------------
// Block sums per target of NDOT compensated sums; the parts of target t land in
// thread t (t < kTB).  `red` holds (kBlock / 32) * kTB * NDOT parts.
template <int NDOT, class AT>
__device__ __forceinline__ void block_tparts(CompSum<AT> (&v)[NDOT], typename CompSum<AT>::Part (&out)[NDOT],
                                             typename CompSum<AT>::Part *red) {
    constexpr int NW = kBlock / 32;
#pragma unroll
    for (int o = 16; o >= kTB; o >>= 1) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) v[k].xor_reduce(o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l < kTB) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) red[(w * kTB + l) * NDOT + k] = v[k].part();
    }
    __syncthreads();
    if (threadIdx.x < kTB) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) {
            CompSum<AT> s;
            for (int q = 0; q < NW; ++q) CompSum<AT>::add_part(s, red[(q * kTB + threadIdx.x) * NDOT + k]);
            out[k] = s.part();
        }
    }
}

// The block's per-target parts go to partials[block][t][k]; returns true in the
// block that arrives last (for all its threads).
template <int NDOT, class Part>
__device__ __forceinline__ bool arrive_last_t(const Part (&mine)[NDOT], Part *partials, unsigned *counter,
                                              const BatchCtl *ctl) {
    __shared__ int last;
    if (threadIdx.x < kTB) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k)
            if (BOK(((int64_t)blockIdx.x * kTB + threadIdx.x) * NDOT + k, ctl->bb.npart, 51))
                partials[((int64_t)blockIdx.x * kTB + threadIdx.x) * NDOT + k] = mine[k];
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = (arrive(counter) == gridDim.x - 1);
    __syncthreads();
    return last != 0;
}

// Per-target fixed-order sums of the grid's parts (last block); target t's
// FP64 totals land in thread t.  `red` holds kBlock * NDOT parts.
template <int NDOT, class AT>
__device__ __forceinline__ void grid_tparts(const typename CompSum<AT>::Part *partials, int nblocks,
                                            double (&out)[NDOT], typename CompSum<AT>::Part *red) {
    const int t = threadIdx.x % kTB, g = threadIdx.x / kTB;
    CompSum<AT> s[NDOT];
    for (int b = g; b < nblocks; b += kTG) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k)
            CompSum<AT>::add_part(s[k], __ldcg(partials + ((int64_t)b * kTB + t) * NDOT + k));
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NDOT; ++k) red[threadIdx.x * NDOT + k] = s[k].part();
    __syncthreads();
    if (threadIdx.x < kTB) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) {
            CompSum<AT> tot;
            for (int q = 0; q < kTG; ++q) CompSum<AT>::add_part(tot, red[(q * kTB + threadIdx.x) * NDOT + k]);
            out[k] = tot.to_double();
        }
    }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// RP[0] = {b, 0}, RP[1] = 0, W = P = 0; per target <r,r>, <mu,r>; start values
template <class FT>
__global__ void __launch_bounds__(kBlock) kb_init(int64_t ldw, int ns, const double *__restrict__ b,
                                                 const double *__restrict__ mu, typename RPair<FT>::T *rp, FT *W,
                                                 FT *P, SolveState *st, BatchCtl *ctl, double *partials,
                                                 unsigned *counter) {
    using R = typename RPair<FT>::T;
    using Part = CompSum<double>::Part;
    __shared__ Part red[kBlock * 2];
    const int64_t m = ldw * kTB;
    CompSum<double> dd[2];
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m; e += (int64_t)gridDim.x * kBlock) {
        const FT rj = (FT)b[e];
        R x;
        x.x = rj;
        x.y = (FT)0;
        rp[e] = x;
        x.x = (FT)0;
        rp[m + e] = x;
        if (W) {   // recurrence form only
            for (int s = 0; s < ns; ++s) {
                W[(int64_t)s * m + e] = (FT)0;
                P[(int64_t)s * m + e] = (FT)0;
            }
        }
        dd[0].add((double)rj * (double)rj);
        dd[1].add(mu[e] * (double)rj);
    }
    Part mine[2];
    block_tparts<2, double>(dd, mine, red);
    if (!arrive_last_t<2>(mine, reinterpret_cast<Part *>(partials), counter, ctl)) return;
    double tot[2];
    grid_tparts<2, double>(reinterpret_cast<const Part *>(partials), gridDim.x, tot, red);
    if (threadIdx.x < kTB) {
        SolveState &S = st[threadIdx.x];
        S.rr = tot[0];
        S.bnorm = sqrt(tot[0]);
        S.inv_bnorm = S.bnorm > 0.0 ? 1.0 / S.bnorm : 0.0;
        S.c = tot[1];
        S.pp = tot[0];
        S.alpha = 0.0;
        S.gamma = 0.0;
        S.gamma_prev = 1.0;
        S.t = 0.0;
        S.k = 0;
        // a non-finite right-hand side stops its target at once, as a breakdown
        S.status = (isfinite(tot[0]) && isfinite(tot[1])) ? SDA_OK : SDA_ERR_BREAKDOWN;
        const bool zero_rhs = !(S.bnorm > 0.0);
        for (int s = 0; s < ns; ++s) {
            ShiftState &h = S.sh[s];
            h.z_prev = 1.0;
            h.z = 1.0;
            h.ratio = 1.0;
            h.g = 0.0;
            h.a = 0.0;
            h.res = zero_rhs ? 0.0 : 1.0;
            h.active = zero_rhs ? 0 : 1;
            h.iters = 0;
        }
        S.nactive = zero_rhs ? 0 : ns;
        S.done = (zero_rhs || S.limit <= 0) ? 1 : 0;
        if (threadIdx.x == 0) *counter = 0u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1;
        for (int t = 0; t < kTB; ++t) all &= st[t].done;
        ctl->k = 0;
        ctl->done = all;
        ctl->status = SDA_OK;
    }
}

// Lanes hold several consecutive targets: one 16-byte access per lane brings
// TPL values of the vector type (4 FP32 / 2 FP64) or PPL {r, p} pairs (2 FP32 /
// 1 FP64); a row or column is served by a group of kTB / TPL (or kTB / PPL)
// lanes, several groups per warp.
template <class FT>
struct BLanes {
    using V = typename Vec16<FT>::T;
    using R = typename RPair<FT>::T;
    static constexpr int TPL = Vec16<FT>::n;                 // targets per lane (vector values)
    static constexpr int LG = kTB / TPL;                     // lanes per group
    static constexpr int PPL = 16 / (int)sizeof(R);          // targets per lane (pairs)
    static constexpr int LGP = kTB / PPL;                    // lanes per group (pairs)
};

// Block sums per target of NDOT compensated sums held TPL targets per thread
// (thread x: targets TPL * (x % (kTB / TPL)) + q); the parts of target t land in
// thread t.  `red` holds (kBlock / 32) * kTB * NDOT parts.
template <int NDOT, int TPL, class AT>
__device__ __forceinline__ void block_tparts_v(CompSum<AT> (&v)[NDOT][TPL], typename CompSum<AT>::Part (&out)[NDOT],
                                               typename CompSum<AT>::Part *red) {
    constexpr int NW = kBlock / 32, LG = kTB / TPL;
#pragma unroll
    for (int o = 16; o >= LG; o >>= 1) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) {
#pragma unroll
            for (int q = 0; q < TPL; ++q) v[k][q].xor_reduce(o);
        }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l < LG) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) {
#pragma unroll
            for (int q = 0; q < TPL; ++q) red[(w * kTB + l * TPL + q) * NDOT + k] = v[k][q].part();
        }
    }
    __syncthreads();
    if (threadIdx.x < kTB) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) {
            CompSum<AT> s;
            for (int q = 0; q < NW; ++q) CompSum<AT>::add_part(s, red[(q * kTB + threadIdx.x) * NDOT + k]);
            out[k] = s.part();
        }
    }
}

// p_k = r_k + alpha_k p_{k-1} of every target, formed once per iteration (the
// row pass then gathers 4 bytes per target and nonzero instead of the pair)
template <class FT>
__global__ void __launch_bounds__(kBlock) kb_formp(int64_t d, int64_t ldw, const typename RPair<FT>::T *__restrict__ pairs,
                                                  FT *__restrict__ p, const SolveState *st, const BatchCtl *ctl) {
    using R = typename RPair<FT>::T;
    if (ctl->done) return;
    const R *__restrict__ a = pairs + (ctl->k & 1) * ldw * kTB;
    const FT al = (FT)st[threadIdx.x % kTB].alpha;
    const int64_t md = d * kTB;
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < md; e += (int64_t)gridDim.x * kBlock) {
        const R x = a[e];
        p[e] = form_p<FT>(x.x, x.y, al);
    }
}

// Targets per thread of the batched row, Laplacian and tail column passes, and
// their resident-block floor: the per-entry work (index, value, bound check) is
// shared by a thread's targets, so FP32 takes eight (two 16-byte gathers; the row
// pass measured 0.81 against 0.98 ms per launch at 2M x 1M with four, at 64
// against 40 registers), FP64 two; the autotuner picks the resident blocks
template <class FT>
struct RowLanes {
    static constexpr int TPL = sizeof(FT) == 4 ? 8 : 2;
    static constexpr int min_blocks = sizeof(FT) == 4 ? 4 : 1;
};

// phase 1: ut[i][t] = (X p_k,t)_i - <mu_t, p_k,t>
template <class VT, class FT>
__global__ void __launch_bounds__(kBlock, RowLanes<FT>::min_blocks) kb_phase1(int64_t n, int64_t ldw, const int64_t *__restrict__ rp,
                                                   const int32_t *__restrict__ col, const VT *__restrict__ val,
                                                   const FT *__restrict__ p, FT *__restrict__ ut,
                                                   const SolveState *st, const BatchCtl *ctl) {
    using V = typename Vec16<FT>::T;
    constexpr int TPL = RowLanes<FT>::TPL, VN = Vec16<FT>::n, NV = TPL / VN, LG = kTB / TPL;
    if (ctl->done) return;
    const int lg = threadIdx.x % LG, t0 = lg * TPL;
    FT c[TPL];
#pragma unroll
    for (int q = 0; q < TPL; ++q) c[q] = (FT)st[t0 + q].c;
    const int64_t g = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / LG;
    const int64_t ng = (int64_t)gridDim.x * (kBlock / LG);
    const int64_t lim = ctl->bb.ldw * kTB;
    const int4 *__restrict__ colq = reinterpret_cast<const int4 *>(col);
    for (int64_t i = g; i < n; i += ng) {
        const int64_t q0 = rp[i] >> 2, q1 = rp[i + 1] >> 2;
        FT acc[TPL];
#pragma unroll
        for (int q = 0; q < TPL; ++q) acc[q] = (FT)0;
        // two quads (eight entries) per step: their indices and values load
        // first, then the eight gathers go out together
        for (int64_t q = q0; q < q1; q += 2) {
            int4 ci[2];
            FT xv[2][4];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                ci[u] = make_int4(0, 0, 0, 0);
#pragma unroll
                for (int e = 0; e < 4; ++e) xv[u][e] = (FT)0;
                if (q + u < q1 && BOK(q + u, ctl->bb.nqx, 11)) {
                    ci[u] = colq[q + u];
                    Quad<VT, FT>::load(val, q + u, xv[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int32_t j = e == 0 ? ci[u].x : e == 1 ? ci[u].y : e == 2 ? ci[u].z : ci[u].w;
                    const int64_t off = (int64_t)j * kTB + t0;
                    if (!BOK(off + TPL - 1, lim, 12)) continue;
                    FT x[TPL];
#pragma unroll
                    for (int v = 0; v < NV; ++v)
                        *reinterpret_cast<V *>(x + v * VN) = *reinterpret_cast<const V *>(p + off + v * VN);
#pragma unroll
                    for (int t = 0; t < TPL; ++t) acc[t] += xv[u][e] * x[t];
                }
            }
        }
        const int64_t io = i * kTB + t0;
        if (BOK(io + TPL - 1, ctl->bb.n8 * kTB, 13)) {
            FT o[TPL];
#pragma unroll
            for (int q = 0; q < TPL; ++q) o[q] = acc[q] - c[q];
#pragma unroll
            for (int v = 0; v < NV; ++v) *reinterpret_cast<V *>(ut + io + v * VN) = *reinterpret_cast<const V *>(o + v * VN);
        }
    }
}

// phase 2: v = omega P_l ut + alpha (D ut - S ut) per target; <ut, v>, 1^T v;
// the last block forms gamma_k per target and the (shift, target) coefficients
template <class FT>
__global__ void __launch_bounds__(kBlock, RowLanes<FT>::min_blocks) kb_phase2(int64_t n, const int64_t *__restrict__ rp,
                                                   const int32_t *__restrict__ col, const FT *__restrict__ sval,
                                                   const FT *__restrict__ ut, const FT *__restrict__ deg,
                                                   const int8_t *__restrict__ ylab, FT *__restrict__ v,
                                                   SolveState *st, BatchCtl *ctl, BatchCoef<FT> *coef, int ns,
                                                   double *partials, unsigned *counter) {
    using V = typename Vec16<FT>::T;
    using Part = typename CompSum<FT>::Part;
    constexpr int TPL = RowLanes<FT>::TPL, VN = Vec16<FT>::n, NV = TPL / VN, LG = kTB / TPL;
    __shared__ Part red[kBlock * 2];
    if (ctl->done) return;
    const int lg = threadIdx.x % LG, t0 = lg * TPL;
    const FT om = (FT)st[0].omega, al = (FT)st[0].alpha_l;
    const int64_t g = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / LG;
    const int64_t ng = (int64_t)gridDim.x * (kBlock / LG);
    const int64_t lim = ctl->bb.n8 * kTB;
    CompSum<FT> dd[2][TPL];
    for (int64_t i = g; i < n; i += ng) {
        const int64_t e0 = rp[i], e1 = rp[i + 1];
        FT acc[TPL];
#pragma unroll
        for (int q = 0; q < TPL; ++q) acc[q] = (FT)0;
        for (int64_t e = e0; e < e1; e += 4) {
            int32_t jj[4];
            FT vv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = e + u < e1 && BOK(e + u, ctl->bb.nnz_s, 21);
                jj[u] = ok ? col[e + u] : 0;
                vv[u] = ok ? sval[e + u] : (FT)0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t off = (int64_t)jj[u] * kTB + t0;
                if (!BOK(off + TPL - 1, lim, 22)) continue;
                FT x[TPL];
#pragma unroll
                for (int w = 0; w < NV; ++w)
                    *reinterpret_cast<V *>(x + w * VN) = *reinterpret_cast<const V *>(ut + off + w * VN);
#pragma unroll
                for (int q = 0; q < TPL; ++q) acc[q] += vv[u] * x[q];
            }
        }
        const int64_t io = i * kTB + t0;
        if (!BOK(io + TPL - 1, lim, 23)) continue;
        FT u[TPL], vo[TPL];
#pragma unroll
        for (int w = 0; w < NV; ++w) *reinterpret_cast<V *>(u + w * VN) = *reinterpret_cast<const V *>(ut + io + w * VN);
        const FT dg = deg[i];
#pragma unroll
        for (int q = 0; q < TPL; ++q) {
            const FT lap = fma(dg, u[q], -acc[q]);
            vo[q] = fma(al, lap, ylab[io + q] != 0 ? om * u[q] : (FT)0);
            dd[0][q].add(u[q] * vo[q]);
            dd[1][q].add(vo[q]);
        }
#pragma unroll
        for (int w = 0; w < NV; ++w) *reinterpret_cast<V *>(v + io + w * VN) = *reinterpret_cast<const V *>(vo + w * VN);
    }
    Part mine[2];
    block_tparts_v<2, TPL, FT>(dd, mine, red);
    if (!arrive_last_t<2>(mine, reinterpret_cast<Part *>(partials), counter, ctl)) return;
    double tot[2];
    grid_tparts<2, FT>(reinterpret_cast<const Part *>(partials), gridDim.x, tot, red);
    if (threadIdx.x < kTB) {
        SolveState &S = st[threadIdx.x];
        if (!S.done) {
            const double pq = tot[0] + S.sigma0 * S.pp;
            if (!(pq > 0.0) || !isfinite(pq)) {
                S.status = SDA_ERR_BREAKDOWN;
                S.done = 1;
                S.gamma = 0.0;
                S.alpha = 0.0;
            } else {
                S.gamma = -S.rr / pq;
                S.t = tot[1];
            }
        }
        if (threadIdx.x == 0) *counter = 0u;
    }
    __syncthreads();
    // zeta_{k+1} / zeta_k and gamma^s_k of every (target, shift) still active
    for (int q = threadIdx.x; q < kTB * ns; q += kBlock) {
        const int tt = q / ns, s = q - tt * ns;
        SolveState &S = st[tt];
        ShiftState &h = S.sh[s];
        BatchCoef<FT> cf;
        cf.z = cf.a = cf.g = (FT)0;
        cf.active = (!S.done && h.active) ? 1 : 0;
        if (cf.active) {
            const double den = S.gamma * S.alpha * (h.z_prev - h.z) + h.z_prev * S.gamma_prev * (1.0 - h.delta * S.gamma);
            const double ratio = h.z_prev * S.gamma_prev / den;
            h.ratio = ratio;
            h.g = S.gamma * ratio;
            cf.z = (FT)h.z;
            cf.a = (FT)h.a;
            cf.g = (FT)h.g;
        }
        if (BOK(s * kTB + tt, kMaxShifts * kTB, 24)) coef[s * kTB + tt] = cf;
    }
}

// phase 3a: s[j][t] = (X^T v_t)_j over the column tiles of the operator's CSC
// (a lane group per column in multi-column tiles; the block's groups share a
// long column's chunk); the four products of a step summed plainly, the steps
// compensated; written as parts
template <class VT, class FT>
__global__ void __launch_bounds__(kBlock, RowLanes<FT>::min_blocks) kb_phase3a(const Tile *__restrict__ tiles, int ntiles,
                                                    const int64_t *__restrict__ cp, const int32_t *__restrict__ row,
                                                    const VT *__restrict__ val, const FT *__restrict__ v,
                                                    typename CompSum<FT>::Part *__restrict__ out,
                                                    typename CompSum<FT>::Part *slots, unsigned *lcount,
                                                    const SplitSeg *__restrict__ splits, const BatchCtl *ctl) {
    using V = typename Vec16<FT>::T;
    using CS = CompSum<FT>;
    using Part = typename CS::Part;
    constexpr int TPL = RowLanes<FT>::TPL, VN = Vec16<FT>::n, NV = TPL / VN, LG = kTB / TPL, GPB = kBlock / LG;
    __shared__ Part red[GPB * kTB];
    __shared__ int last;
    if (ctl->done) return;
    const int lg = threadIdx.x % LG, g = threadIdx.x / LG, t0 = lg * TPL;
    const int64_t lim = ctl->bb.n8 * kTB;
    // eight entries (stride `step`) per round: their indices and values load
    // first, then the gathers go out together; each group of four entries is
    // summed, then added to the compensated sums
    auto dot = [&](int64_t e0, int64_t e1, int64_t step, CS (&acc)[TPL]) {
        for (int64_t e = e0; e < e1; e += 8 * step) {
            int32_t ii[8];
            FT vv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const bool ok = e + u * step < e1 && BOK(e + u * step, ctl->bb.nnz_x, 31);
                ii[u] = ok ? row[e + u * step] : 0;
                vv[u] = ok ? (FT)Val<VT>::get(val, e + u * step) : (FT)0;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h == 1 && e + 4 * step >= e1) break;
                FT sum[TPL];
#pragma unroll
                for (int q = 0; q < TPL; ++q) sum[q] = (FT)0;
#pragma unroll
                for (int u = 4 * h; u < 4 * h + 4; ++u) {
                    const int64_t off = (int64_t)ii[u] * kTB + t0;
                    if (!BOK(off + TPL - 1, lim, 32)) continue;
                    FT x[TPL];
#pragma unroll
                    for (int w = 0; w < NV; ++w)
                        *reinterpret_cast<V *>(x + w * VN) = *reinterpret_cast<const V *>(v + off + w * VN);
#pragma unroll
                    for (int q = 0; q < TPL; ++q) sum[q] += vv[u] * x[q];
                }
#pragma unroll
                for (int q = 0; q < TPL; ++q) acc[q].add(sum[q]);
            }
        }
    };
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const Tile tl = tiles[tile];
        if (tl.lanes > 0) {
            // columns go to lane groups from a starting group that moves from
            // tile to tile (23 is odd: every residue in turn), so that tiles of
            // few columns do not always load the same groups
            const int nseg = tl.seg1 - tl.seg0;
            const int rot = (it * 23 + blockIdx.x) % GPB;
            for (int sgi = (g - rot + GPB) % GPB; sgi < nseg; sgi += GPB) {
                const int64_t j = tl.seg0 + sgi;
                if (!BOK(j, ctl->bb.d, 33)) continue;
                CS acc[TPL];
                dot(cp[j], cp[j + 1], 1, acc);
#pragma unroll
                for (int q = 0; q < TPL; ++q) out[j * kTB + t0 + q] = acc[q].part();
            }
            continue;
        }
        CS acc[TPL];
        dot(tl.nz0 + g, tl.nz1, GPB, acc);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TPL; ++q) red[g * kTB + t0 + q] = acc[q].part();
        __syncthreads();
        Part part{};
        if (threadIdx.x < kTB) {
            CS tot;
            for (int q = 0; q < GPB; ++q) CS::add_part(tot, red[q * kTB + threadIdx.x]);
            part = tot.part();
        }
        if (tl.slot < 0) {
            if (threadIdx.x < kTB && BOK(tl.seg0, ctl->bb.d, 34)) out[(int64_t)tl.seg0 * kTB + threadIdx.x] = part;
            continue;
        }
        if (!BOK(tl.slot, ctl->bb.nslots, 35) || !BOK(tl.lseg, ctl->bb.nsplits, 36)) {
            __syncthreads();
            continue;
        }
        if (threadIdx.x < kTB) {
            slots[(int64_t)tl.slot * kTB + threadIdx.x] = part;
            __threadfence();
        }
        __syncthreads();
        if (threadIdx.x == 0) last = (arrive(&lcount[tl.lseg]) == (unsigned)splits[tl.lseg].nchunks - 1u);
        __syncthreads();
        if (last && threadIdx.x < kTB) {
            const SplitSeg sp = splits[tl.lseg];
            CS tot;
            for (int q = 0; q < sp.nchunks; ++q) CS::add_part(tot, __ldcg(slots + (int64_t)(sp.slot0 + q) * kTB + threadIdx.x));
            out[(int64_t)tl.seg0 * kTB + threadIdx.x] = tot.part();
            if (threadIdx.x == 0) lcount[tl.lseg] = 0u;
        }
        __syncthreads();
    }
}

// phase 3a, head columns: for every range r of kHeadRows rows the block stages
// the range's slice of V ([rows][kTB], the vector type) in shared memory; lane
// groups then take the head columns in turn and sum x_ij V[i] over the column's
// entries in the range (quads of 16-bit local rows, gathers from shared memory;
// each quad summed plainly, the quads compensated) into hp[r][h][kTB]
template <class VT, class FT>
__global__ void __launch_bounds__(kBlock) kb_head3a(int64_t n, int nr, int H, int nsplit,
                                                   const int64_t *__restrict__ cp, const uint16_t *__restrict__ idx,
                                                   const VT *__restrict__ val, const FT *__restrict__ v,
                                                   typename CompSum<FT>::Part *__restrict__ hp, const BatchCtl *ctl) {
    using L = BLanes<FT>;
    using V = typename L::V;
    using CS = CompSum<FT>;
    constexpr int TPL = L::TPL, LG = L::LG, GPB = kBlock / LG;
    extern __shared__ __align__(16) unsigned char kh_dyn[];
    FT *vs = reinterpret_cast<FT *>(kh_dyn);
    if (ctl->done) return;
    const int lg = threadIdx.x % LG, g = threadIdx.x / LG, t0 = lg * TPL;
    const uint2 *__restrict__ idxq = reinterpret_cast<const uint2 *>(idx);
    // work items (range r, slice c of the head columns), nsplit slices per range
    const int hs = (H + nsplit - 1) / nsplit;
    for (int item = blockIdx.x; item < nr * nsplit; item += gridDim.x) {
        const int r = item / nsplit, c0 = (item - r * nsplit) * hs, c1 = min(H, c0 + hs);
        const int64_t row0 = (int64_t)r * kHeadRows;
        const int rows = (int)min((int64_t)kHeadRows, n - row0);
        __syncthreads();
        {
            const V *__restrict__ src = reinterpret_cast<const V *>(v + row0 * kTB);
            V *dst = reinterpret_cast<V *>(vs);
            const int nvec = rows * (kTB / TPL);
            for (int q = threadIdx.x; q < nvec; q += kBlock) dst[q] = src[q];
        }
        __syncthreads();
        const int64_t *__restrict__ c = cp + (int64_t)r * (H + 1);
        for (int h = c0 + g; h < c1; h += GPB) {
            const int64_t q0 = c[h] >> 2, q1 = c[h + 1] >> 2;
            CS acc[TPL];
            // four quads per step: their indices and values load first (independent
            // global loads in flight), then the sixteen gathers from shared memory
            for (int64_t q = q0; q < q1; q += 4) {
                uint2 ii[4];
                FT xv[4][4];
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    if (q + w < q1) {
                        ii[w] = idxq[q + w];
                        Quad<VT, FT>::load(val, q + w, xv[w]);
                    } else {
                        ii[w] = make_uint2(0u, 0u);
#pragma unroll
                        for (int k = 0; k < 4; ++k) xv[w][k] = (FT)0;
                    }
                }
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const int li[4] = {(int)(ii[w].x & 0xffffu), (int)(ii[w].x >> 16), (int)(ii[w].y & 0xffffu),
                                       (int)(ii[w].y >> 16)};
                    FT sum[TPL];
#pragma unroll
                    for (int u = 0; u < TPL; ++u) sum[u] = (FT)0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        FT x[TPL];
                        *reinterpret_cast<V *>(x) = *reinterpret_cast<const V *>(vs + li[k] * kTB + t0);
#pragma unroll
                        for (int u = 0; u < TPL; ++u) sum[u] += xv[w][k] * x[u];
                    }
#pragma unroll
                    for (int u = 0; u < TPL; ++u) acc[u].add(sum[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < TPL; ++u) hp[((int64_t)r * H + h) * kTB + t0 + u] = acc[u].part();
        }
    }
}

// out[e] = sum over the ranges r of hp[r][e] for e < m (fixed order: warp w adds
// the ranges r = w mod 8, then the eight warps' sums in order)
template <class FT>
__global__ void __launch_bounds__(kBlock) kb_head_reduce(int nr, int64_t m, const typename CompSum<FT>::Part *__restrict__ hp,
                                                        typename CompSum<FT>::Part *__restrict__ out,
                                                        const BatchCtl *ctl) {
    using CS = CompSum<FT>;
    using Part = typename CS::Part;
    constexpr int NW = kBlock / 32;
    __shared__ Part red[kBlock];
    if (ctl->done) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t e0 = (int64_t)blockIdx.x * 32; e0 < m; e0 += (int64_t)gridDim.x * 32) {
        const int64_t e = e0 + lane;
        CS acc;
        if (e < m)
            for (int r = w; r < nr; r += NW) CS::add_part(acc, hp[(int64_t)r * m + e]);
        __syncthreads();
        red[threadIdx.x] = acc.part();
        __syncthreads();
        if (w == 0 && e < m) {
            CS tot;
#pragma unroll
            for (int q = 0; q < NW; ++q) CS::add_part(tot, red[q * 32 + lane]);
            out[e] = tot.part();
        }
    }
}

// ---------------------------------------------------------------------------
// Exact fixed-point X passes of the FP64 block utilities
// ---------------------------------------------------------------------------
// GB300 runs FP64 arithmetic at a small fraction of its FP32 and integer rates,
// and an FP64 pass over X costs one FP64 multiply-add per lane and nonzero. When
// the values of X are small integers times one power of two (binary and count
// data: x = x_int 2^-sx, |x_int| < 2^bx), the X passes run on integers instead:
// a lane's vector z is scaled to z_fx = round(z 2^k) with |z_fx| <= 2^(62 - bx),
// k set by the lane's largest |z|, and stored as two 32-bit halves z_fx =
// hi 2^31 + lo (0 <= lo < 2^31). Each product is two 32 x 32 -> 64-bit
// multiply-adds into a 64-bit sum of the lo products and one of the hi products
// (exact while a sum has fewer than 2^(32 - bx) terms), combined exactly in 128
// bits and rounded to FP64 once per result. The only other error is the
// rounding of z to multiples of 2^-k: per entry at most 2^-(k+1) sum_j |x_ij|,
// i.e. about 2^(bx - 63) max|z| sum_j |x_ij|, no larger than the rounding of an
// FP64 sum of the same terms.
using i128 = __int128;

// The row and tail column passes gather all 16 lanes of a row of z_fx (128 bytes,
// one pass; measured against two passes over planes of 8 lanes, 64-byte rows,
// at 2M x 1M: 988 against 1011 ms per 32-target sweep with its residual check);
// the head pass stages 8 lanes of a range at a time (96 KB of shared memory)
constexpr int kFxNT = 16;                 // lanes per row of the scaled block ([len][kFxNT] planes)
constexpr int kFxHNT = 8;                 // lanes a head work item stages
constexpr int kFxTPL = 4;                 // lanes per thread in the fixed-point passes
constexpr int kFxNonFinite = -(1 << 30);  // scale exponent of a lane holding a non-finite value

__device__ __forceinline__ double i128_to_double(i128 a) {
    const long long hi = (long long)(a >> 64);
    const unsigned long long lo = (unsigned long long)a;
    if (hi == ((long long)lo >> 63)) return (double)(long long)lo;   // fits in 64 bits: one rounding
    return (double)hi * 18446744073709551616.0 + (double)lo;          // |a| >= 2^63: within 2^-52 |a|
}

// a result scaled back: a 2^-(k + sx), NaN for a non-finite lane (2^-(k + sx) built
// from its exponent bits when it is a normal double, as it is for every vector
// whose largest entry lies between 2^-950 and 2^1000)
__device__ __forceinline__ double fx_value(i128 a, int k, int sx) {
    if (k == kFxNonFinite) return (double)NAN;
    const int e = k + sx;
    if (e > -1000 && e < 1000) return i128_to_double(a) * __longlong_as_double((long long)(1023 - e) << 52);
    return ldexp(i128_to_double(a), -e);
}

// x_int = x 2^sx of a stored value read as XF (exact: x has few significant bits)
template <class XF>
__device__ __forceinline__ int fx_int(XF x, XF xs) {
    return (int)(x * xs);
}

// the two partial sums of a lane: sum x_int lo and sum x_int hi
struct FxAcc {
    long long lo = 0, hi = 0;
    __device__ __forceinline__ void add(int x, int zlo, int zhi) {
        lo += (long long)x * (long long)zlo;
        hi += (long long)x * (long long)zhi;
    }
    __device__ __forceinline__ i128 total() const { return ((i128)hi << 31) + (i128)lo; }
};

// amax[l] = max over i < len of |src[i][l]| as its bit pattern (non-negative
// doubles order as their bits; a NaN or infinity is at least 0x7ff0...)
__global__ void __launch_bounds__(kBlock) kb_absmax_lanes(int64_t len, const double *__restrict__ src,
                                                         unsigned long long *amax) {
    unsigned long long m = 0;
    const int64_t total = len * kTB;
    // kBlock and the grid stride are multiples of kTB: thread x always sees lane x % kTB
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < total; e += (int64_t)gridDim.x * kBlock) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(src[e]));
        m = b > m ? b : m;
    }
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, 16);
    m = o > m ? o : m;
    if ((threadIdx.x & 31) < kTB) atomicMax(amax + threadIdx.x % kTB, m);
}

// scale exponent k of a lane from its amax: |z| 2^k < 2^(62 - bx)
__device__ __forceinline__ int fx_exp(unsigned long long amax_bits, int bx) {
    if (amax_bits >= 0x7ff0000000000000ull) return kFxNonFinite;
    if (amax_bits == 0ull) return 0;
    int e = 0;
    frexp(__longlong_as_double((long long)amax_bits), &e);   // max |z| < 2^e
    return 62 - bx - e;
}

// dst planes [kTB / kFxNT][len][kFxNT] of round(src[i][l] 2^k_l) as {lo, hi}
// halves; k_l to kexp
__global__ void __launch_bounds__(kBlock) kb_to_fixed(int64_t len, const double *__restrict__ src,
                                                     const unsigned long long *__restrict__ amax, int bx,
                                                     int2 *__restrict__ dst, int *kexp) {
    const int l = threadIdx.x % kTB;
    const int k = fx_exp(amax[l], bx);
    if (blockIdx.x == 0 && threadIdx.x < kTB) kexp[threadIdx.x] = k;
    const int64_t total = len * kTB;
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < total; e += (int64_t)gridDim.x * kBlock) {
        const int64_t i = e / kTB;
        const long long q = k == kFxNonFinite ? 0ll : llrint(ldexp(src[e], k));   // |q| <= 2^(62 - bx)
        dst[(int64_t)(l / kFxNT) * len * kFxNT + i * kFxNT + (l % kFxNT)] =
            make_int2((int)(q & 0x7fffffffll), (int)(q >> 31));
    }
}

// lowest and highest set-bit exponents of the nonzero values of X (for x_int):
// out[0] = min E, out[1] = max T over x = M 2^E (M odd), 2^T <= |x| < 2^(T+1);
// out[2] = 1 if a value is not finite
template <class VT>
__global__ void __launch_bounds__(kBlock) kb_fx_scan(int64_t nnz, const VT *__restrict__ val, int *out) {
    int lo = 1 << 30, hi = -(1 << 30), bad = 0;
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * kBlock) {
        const double x = (double)Val<VT>::get(val, e);
        if (x == 0.0) continue;
        if (!isfinite(x)) {
            bad = 1;
            continue;
        }
        int ex = 0;
        const double m = frexp(fabs(x), &ex);   // |x| = m 2^ex, m in [0.5, 1)
        const unsigned long long M = (unsigned long long)ldexp(m, 53);
        lo = min(lo, ex - 53 + (__ffsll((long long)M) - 1));
        hi = max(hi, ex - 1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(out + 0, lo);
        atomicMax(out + 1, hi);
        if (bad) atomicOr(out + 2, 1);
    }
}

// four lanes' products with one value: z_fx halves of lanes t .. t + 3 at p
// ({lo, hi} pairs, 32-byte aligned)
__device__ __forceinline__ void fx_add4(FxAcc (&acc)[4], int x, const int2 *p) {
    const int4 a = reinterpret_cast<const int4 *>(p)[0];
    const int4 b = reinterpret_cast<const int4 *>(p)[1];
    acc[0].add(x, a.x, a.y);
    acc[1].add(x, a.z, a.w);
    acc[2].add(x, b.x, b.y);
    acc[3].add(x, b.z, b.w);
}

// phase 1 in fixed point: ut[i][t] = (X w_t)_i - c_t for the kFxNT lanes
// t = lane0 .., gathered from one plane wp ([ldw][kFxNT]) of w_fx; four lanes per thread
template <class VT>
__global__ void __launch_bounds__(kBlock, 3) kb_phase1_fx(int64_t n, const int64_t *__restrict__ rp,
                                                         const int32_t *__restrict__ col, const VT *__restrict__ val,
                                                         const int2 *__restrict__ wp, double *__restrict__ ut,
                                                         const SolveState *st, const BatchCtl *ctl, int lane0, int sx,
                                                         const int *__restrict__ kexp) {
    using XF = std::conditional_t<std::is_same<VT, double>::value, double, float>;
    constexpr int TPL = kFxTPL, LG = kFxNT / TPL;
    if (ctl->done) return;
    const int lg = threadIdx.x % LG, t0 = lg * TPL;
    double c[TPL];
    int kq[TPL];
#pragma unroll
    for (int q = 0; q < TPL; ++q) {
        c[q] = st[lane0 + t0 + q].c;
        kq[q] = kexp[lane0 + t0 + q];
    }
    const XF xs = (XF)(1ll << sx);
    const int64_t g = ((int64_t)blockIdx.x * kBlock + threadIdx.x) / LG;
    const int64_t ng = (int64_t)gridDim.x * (kBlock / LG);
    const int64_t lim = ctl->bb.ldw * kFxNT;
    const int4 *__restrict__ colq = reinterpret_cast<const int4 *>(col);
    for (int64_t i = g; i < n; i += ng) {
        const int64_t q0 = rp[i] >> 2, q1 = rp[i + 1] >> 2;
        FxAcc acc[TPL];
        for (int64_t q = q0; q < q1; q += 2) {
            int4 ci[2];
            int xi[2][4];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                ci[u] = make_int4(0, 0, 0, 0);
#pragma unroll
                for (int e = 0; e < 4; ++e) xi[u][e] = 0;
                if (q + u < q1 && BOK(q + u, ctl->bb.nqx, 60)) {
                    ci[u] = colq[q + u];
                    XF xv[4];
                    Quad<VT, XF>::load(val, q + u, xv);
#pragma unroll
                    for (int e = 0; e < 4; ++e) xi[u][e] = fx_int(xv[e], xs);
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int32_t j = e == 0 ? ci[u].x : e == 1 ? ci[u].y : e == 2 ? ci[u].z : ci[u].w;
                    const int64_t off = (int64_t)j * kFxNT + t0;
                    if (!BOK(off + TPL - 1, lim, 61)) continue;
                    fx_add4(acc, xi[u][e], wp + off);
                }
            }
        }
        const int64_t io = i * kTB + lane0 + t0;
        if (BOK(io + TPL - 1, ctl->bb.n8 * kTB, 62)) {
            double o[TPL];
#pragma unroll
            for (int q = 0; q < TPL; ++q) o[q] = fx_value(acc[q].total(), kq[q], sx) - c[q];
            reinterpret_cast<double2 *>(ut + io)[0] = make_double2(o[0], o[1]);
            reinterpret_cast<double2 *>(ut + io)[1] = make_double2(o[2], o[3]);
        }
    }
}

// head columns in fixed point: as kb_head3a, the range slice of kFxHNT lanes of
// v_fx (lanes hf * kFxHNT .., from the planes) staged in shared memory; hp[r][h][t]
// gets the range's sum scaled back to FP64; two lanes per thread (measured faster
// here than four: 1.90 against 2.16 ms per launch at 2M x 1M)
template <class VT>
__global__ void __launch_bounds__(kBlock) kb_head3a_fx(int64_t n, int64_t n8, int nr, int H, int nsplit,
                                                      const int64_t *__restrict__ cp, const uint16_t *__restrict__ idx,
                                                      const VT *__restrict__ val, const int2 *__restrict__ vpl,
                                                      double *__restrict__ hp, const BatchCtl *ctl, int sx,
                                                      const int *__restrict__ kexp) {
    using XF = std::conditional_t<std::is_same<VT, double>::value, double, float>;
    constexpr int NH = kTB / kFxHNT, TPL = 2, LG = kFxHNT / TPL, GPB = kBlock / LG, VPR = kFxHNT / 2;
    extern __shared__ __align__(16) unsigned char khx_dyn[];
    int2 *vs = reinterpret_cast<int2 *>(khx_dyn);
    if (ctl->done) return;
    const int lg = threadIdx.x % LG, g = threadIdx.x / LG, t0 = lg * TPL;
    const uint2 *__restrict__ idxq = reinterpret_cast<const uint2 *>(idx);
    const XF xs = (XF)(1ll << sx);
    const int hs = (H + nsplit - 1) / nsplit;
    for (int item = blockIdx.x; item < nr * nsplit * NH; item += gridDim.x) {
        const int r = item / (nsplit * NH), rem = item - r * nsplit * NH;
        const int sl = rem / NH, hf = rem - sl * NH;
        const int c0 = sl * hs, c1 = min(H, c0 + hs);
        const int64_t row0 = (int64_t)r * kHeadRows;
        const int rows = (int)min((int64_t)kHeadRows, n - row0);
        __syncthreads();
        {
            // lanes hf * kFxHNT .. of rows row0 ..: plane pl at offset o within its rows
            const int pl = (hf * kFxHNT) / kFxNT, o = (hf * kFxHNT) % kFxNT;
            const int2 *__restrict__ base = vpl + ((int64_t)pl * n8 + row0) * kFxNT + o;
            int4 *dst = reinterpret_cast<int4 *>(vs);
            const int nvec = rows * VPR;
            for (int q = threadIdx.x; q < nvec; q += kBlock) {
                const int i = q / VPR;
                dst[q] = reinterpret_cast<const int4 *>(base + (int64_t)i * kFxNT)[q - i * VPR];
            }
        }
        __syncthreads();
        int kq[TPL];
#pragma unroll
        for (int u = 0; u < TPL; ++u) kq[u] = kexp[hf * kFxHNT + t0 + u];
        const int64_t *__restrict__ c = cp + (int64_t)r * (H + 1);
        for (int h = c0 + g; h < c1; h += GPB) {
            const int64_t q0 = c[h] >> 2, q1 = c[h + 1] >> 2;
            FxAcc acc[TPL];
            for (int64_t q = q0; q < q1; q += 4) {
                uint2 ii[4];
                int xi[4][4];
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    if (q + w < q1) {
                        ii[w] = idxq[q + w];
                        XF xv[4];
                        Quad<VT, XF>::load(val, q + w, xv);
#pragma unroll
                        for (int k = 0; k < 4; ++k) xi[w][k] = fx_int(xv[k], xs);
                    } else {
                        ii[w] = make_uint2(0u, 0u);
#pragma unroll
                        for (int k = 0; k < 4; ++k) xi[w][k] = 0;
                    }
                }
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const int li[4] = {(int)(ii[w].x & 0xffffu), (int)(ii[w].x >> 16), (int)(ii[w].y & 0xffffu),
                                       (int)(ii[w].y >> 16)};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int4 x = *reinterpret_cast<const int4 *>(vs + li[k] * kFxHNT + t0);
                        acc[0].add(xi[w][k], x.x, x.y);
                        acc[1].add(xi[w][k], x.z, x.w);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < TPL; ++u)
                hp[((int64_t)r * H + h) * kTB + hf * kFxHNT + t0 + u] = fx_value(acc[u].total(), kq[u], sx);
        }
    }
}

// tail columns in fixed point: as kb_phase3a for the kFxNT lanes t = lane0 ..,
// gathered from one plane v ([n8][kFxNT]) of v_fx; the block and split-column
// sums stay in 128-bit integers (slots: one i128 per lane) until the column's
// total is scaled back to FP64
template <class VT>
__global__ void __launch_bounds__(kBlock, 3) kb_phase3a_fx(const Tile *__restrict__ tiles, int ntiles,
                                                          const int64_t *__restrict__ cp,
                                                          const int32_t *__restrict__ row, const VT *__restrict__ val,
                                                          const int2 *__restrict__ v, double *__restrict__ out,
                                                          i128 *slots, unsigned *lcount,
                                                          const SplitSeg *__restrict__ splits, const BatchCtl *ctl,
                                                          int lane0, int sx, const int *__restrict__ kexp) {
    using XF = std::conditional_t<std::is_same<VT, double>::value, double, float>;
    constexpr int TPL = kFxTPL, LG = kFxNT / TPL, GPB = kBlock / LG;
    __shared__ i128 red[GPB * kFxNT];
    __shared__ int last;
    if (ctl->done) return;
    const int lg = threadIdx.x % LG, g = threadIdx.x / LG, t0 = lg * TPL;
    const int64_t lim = ctl->bb.n8 * kFxNT;
    const XF xs = (XF)(1ll << sx);
    int kq[TPL];
#pragma unroll
    for (int u = 0; u < TPL; ++u) kq[u] = kexp[lane0 + t0 + u];
    const int lt = lane0 + (int)(threadIdx.x % kFxNT);   // the lane thread x < kFxNT reduces
    const int kr = kexp[lt];
    // eight entries (stride `step`) per round: indices and values first, then the gathers
    auto dot = [&](int64_t e0, int64_t e1, int64_t step, FxAcc (&acc)[TPL]) {
        for (int64_t e = e0; e < e1; e += 8 * step) {
            int32_t ii[8];
            int xi[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const bool ok = e + u * step < e1 && BOK(e + u * step, ctl->bb.nnz_x, 63);
                ii[u] = ok ? row[e + u * step] : 0;
                xi[u] = ok ? fx_int((XF)Val<VT>::get(val, e + u * step), xs) : 0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t off = (int64_t)ii[u] * kFxNT + t0;
                if (!BOK(off + TPL - 1, lim, 64)) continue;
                fx_add4(acc, xi[u], v + off);
            }
        }
    };
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const Tile tl = tiles[tile];
        if (tl.lanes > 0) {
            const int nseg = tl.seg1 - tl.seg0;
            const int rot = (it * 23 + blockIdx.x) % GPB;
            for (int sgi = (g - rot + GPB) % GPB; sgi < nseg; sgi += GPB) {
                const int64_t j = tl.seg0 + sgi;
                if (!BOK(j, ctl->bb.d, 65)) continue;
                FxAcc acc[TPL];
                dot(cp[j], cp[j + 1], 1, acc);
#pragma unroll
                for (int q = 0; q < TPL; ++q) out[j * kTB + lane0 + t0 + q] = fx_value(acc[q].total(), kq[q], sx);
            }
            continue;
        }
        FxAcc acc[TPL];
        dot(tl.nz0 + g, tl.nz1, GPB, acc);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TPL; ++q) red[g * kFxNT + t0 + q] = acc[q].total();
        __syncthreads();
        i128 part = 0;
        if (threadIdx.x < kFxNT)
            for (int q = 0; q < GPB; ++q) part += red[q * kFxNT + threadIdx.x];
        if (tl.slot < 0) {
            if (threadIdx.x < kFxNT && BOK(tl.seg0, ctl->bb.d, 66))
                out[(int64_t)tl.seg0 * kTB + lt] = fx_value(part, kr, sx);
            continue;
        }
        if (!BOK(tl.slot, ctl->bb.nslots, 67) || !BOK(tl.lseg, ctl->bb.nsplits, 68)) {
            __syncthreads();
            continue;
        }
        if (threadIdx.x < kFxNT) {
            slots[(int64_t)tl.slot * kTB + lt] = part;
            __threadfence();
        }
        __syncthreads();
        if (threadIdx.x == 0) last = (arrive(&lcount[tl.lseg]) == (unsigned)splits[tl.lseg].nchunks - 1u);
        __syncthreads();
        if (last && threadIdx.x < kFxNT) {
            const SplitSeg sp = splits[tl.lseg];
            i128 tot = 0;
            for (int q = 0; q < sp.nchunks; ++q) {
                const long long *p2 = reinterpret_cast<const long long *>(slots + (int64_t)(sp.slot0 + q) * kTB + lt);
                tot += ((i128)__ldcg(p2 + 1) << 64) | (i128)(unsigned long long)__ldcg(p2);
            }
            out[(int64_t)tl.seg0 * kTB + lt] = fx_value(tot, kr, sx);
            if (threadIdx.x == 0) lcount[tl.lseg] = 0u;
        }
        __syncthreads();
    }
}

// phase 3b: base recurrence per (feature, target), shift-state stream over the
// shifts some target still updates, per-target dots; the last block forms
// alpha_{k+1}, the shift coefficients and the stop tests of every target
template <class FT>
__global__ void __launch_bounds__(kBlock) kb_phase3b(int64_t d, int64_t ldw, int ns,
                                                    const typename CompSum<FT>::Part *__restrict__ s,
                                                    typename RPair<FT>::T *__restrict__ pairs, FT *__restrict__ W,
                                                    FT *__restrict__ P, SolveState *st, BatchCtl *ctl,
                                                    const BatchCoef<FT> *__restrict__ coef,
                                                    const float *__restrict__ mu32, const double *__restrict__ mu64,
                                                    double *partials, unsigned *counter, BasisView<FT> bvw) {
    using R = typename RPair<FT>::T;
    using Part = typename CompSum<FT>::Part;
    __shared__ Part red[kBlock * 3];
    extern __shared__ __align__(16) unsigned char kb3b_dyn[];   // the ns x kTB coefficients
    BatchCoef<FT> *cf = reinterpret_cast<BatchCoef<FT> *>(kb3b_dyn);
    __shared__ int any[kMaxShifts];
    __shared__ int s_act[kMaxShifts];
    __shared__ int s_nact;
    __shared__ FT s_al[kTB];
    __shared__ double s_gam[kTB], s_t[kTB];
    __shared__ float s_gh[kTB], s_gl[kTB], s_tf[kTB];
    __shared__ float s_sh[kTB], s_sl[kTB];   // each lane's base shift sigma0 as an FP32 pair
    __shared__ double s_sigma0[kTB];
    __shared__ double s_anw[kTB], s_rn[kTB];
    __shared__ int s_exact[kTB];
    if (ctl->done) return;
    if (threadIdx.x < kTB) {
        const SolveState &S = st[threadIdx.x];
        s_al[threadIdx.x] = (FT)S.alpha;
        s_gam[threadIdx.x] = S.gamma;
        s_t[threadIdx.x] = S.t;
        split_f32(S.gamma, s_gh[threadIdx.x], s_gl[threadIdx.x]);
        s_tf[threadIdx.x] = (float)S.t;
        s_sigma0[threadIdx.x] = S.sigma0;
        split_f32(S.sigma0, s_sh[threadIdx.x], s_sl[threadIdx.x]);
    }
    for (int q = threadIdx.x; q < ns * kTB; q += kBlock) cf[q] = coef[q];
    if (threadIdx.x < ns) any[threadIdx.x] = 0;
    __syncthreads();
    for (int q = threadIdx.x; q < ns * kTB; q += kBlock)
        if (cf[q].active) any[q / kTB] = 1;
    __syncthreads();
    const int64_t m = ldw * kTB;
    const int par = ctl->k & 1;
    const R *__restrict__ a = pairs + par * m;
    R *__restrict__ an_ = pairs + (par ^ 1) * m;
    const int64_t tid = (int64_t)blockIdx.x * kBlock + threadIdx.x, nthr = (int64_t)gridDim.x * kBlock;
    const int t = threadIdx.x % kTB;
    CompSum<FT> dd[3];
    const int64_t md = d * kTB;
    // stored-basis form: r_k of every lane goes to basis slot k
    FT *__restrict__ bslot = bvw.tab ? bvw.tab[ctl->k / bvw.per_chunk] + (int64_t)(ctl->k % bvw.per_chunk) * m : nullptr;
    for (int64_t e = tid; e < md; e += nthr) {
        if (!BOK(e, ctl->bb.ldw * kTB, 41)) continue;
        const R x = a[e];
        if (bslot) bslot[e] = x.x;
        const FT pk = form_p<FT>(x.x, x.y, s_al[t]);
        CompSum<FT> sj;
        CompSum<FT>::add_part(sj, s[e]);
        FT rnj, mj;
        if constexpr (std::is_same<FT, float>::value) {
            mj = mu32[e];
            rnj = base_step_f32v(x.x, pk, sj.h, sj.l, mj, s_sh[t], s_sl[t], s_tf[t], s_gh[t], s_gl[t]);
        } else {
            const double m64 = mu64[e];
            mj = (FT)m64;
            const double qj = (double)sj.value() - m64 * s_t[t] + s_sigma0[t] * (double)pk;
            rnj = (FT)((double)x.x + s_gam[t] * qj);
        }
        R y;
        y.x = rnj;
        y.y = pk;
        an_[e] = y;
        dd[0].add(rnj * rnj);
        dd[1].add(mj * rnj);
        dd[2].add(rnj * pk);
    }
    // shift state: P^s_k = zeta r_k + alpha^s P^s_{k-1}; W^s_{k+1} = W^s_k - gamma^s P^s_k
    // (targets whose shift stopped keep their values).  Items i = q * nch + c over
    // the shifts some target still updates (slot q) and 16-byte chunks c of VW
    // consecutive targets of one feature; (q, c) advance by (nthr / nch, nthr %
    // nch), two items per thread in flight.  The stored-basis form skips it.
    if (!bvw.tab) {
        using V = typename Vec16<FT>::T;
        constexpr int VW = Vec16<FT>::n;
        constexpr int UNROLL = 2;
        if (threadIdx.x == 0) {
            int na = 0;
            for (int sh = 0; sh < ns; ++sh)
                if (any[sh]) s_act[na++] = sh;
            s_nact = na;
        }
        __syncthreads();
        const int nch = (int)(m / VW), nact = s_nact;
        int q = (int)(tid / nch), c = (int)(tid - (int64_t)q * nch);
        const int sq = (int)(nthr / nch), sc = (int)(nthr - (int64_t)sq * nch);
        while (q < nact) {
            FT r[UNROLL][VW];
            V pv[UNROLL], wv[UNROLL];
            int64_t off[UNROLL], e0[UNROLL];
            int sh_[UNROLL];
            bool ok[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                ok[u] = q < nact;
                sh_[u] = ok[u] ? s_act[q] : 0;
                e0[u] = (int64_t)c * VW;
                off[u] = (int64_t)sh_[u] * m + e0[u];
                ok[u] = ok[u] && BOK(e0[u] + VW - 1, ctl->bb.ldw * kTB, 42);
                if (ok[u]) {
                    load_r(a, e0[u], r[u]);
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
                if (!ok[u]) continue;
                const BatchCoef<FT> *cb = cf + sh_[u] * kTB + (int)(e0[u] % kTB);
#pragma unroll
                for (int v = 0; v < VW; ++v) {
                    const BatchCoef<FT> cu = cb[v];
                    if (!cu.active) continue;
                    const FT pn = cu.z * r[u][v] + cu.a * v16_get(pv[u], v);
                    v16_set(pv[u], v, pn);
                    v16_set(wv[u], v, v16_get(wv[u], v) - cu.g * pn);
                }
                *reinterpret_cast<V *>(P + off[u]) = pv[u];
                *reinterpret_cast<V *>(W + off[u]) = wv[u];
            }
        }
    }
    Part mine[3];
    block_tparts<3, FT>(dd, mine, red);
    if (!arrive_last_t<3>(mine, reinterpret_cast<Part *>(partials), counter, ctl)) return;
    double tot[3];
    grid_tparts<3, FT>(reinterpret_cast<const Part *>(partials), gridDim.x, tot, red);
    if (threadIdx.x < kTB) {
        SolveState &S = st[threadIdx.x];
        s_anw[threadIdx.x] = 0.0;
        s_rn[threadIdx.x] = 0.0;
        s_exact[threadIdx.x] = 0;
        if (!S.done) {
            const double rr_new = tot[0];
            // an exactly vanished residual ends the lane's run (a fixed-iteration run
            // would otherwise go on with p = 0 and divide by <p, (B + sigma0) p> = 0)
            s_exact[threadIdx.x] = rr_new == 0.0;
            const double anw = rr_new / S.rr;
            const double c_new = tot[1] + anw * S.c;
            const double pp_new = rr_new + 2.0 * anw * tot[2] + anw * anw * S.pp;
            if (!isfinite(rr_new) || !isfinite(anw)) S.status = SDA_ERR_BREAKDOWN;
            if (bvw.lz) bvw.lz[(int64_t)S.k * kTB + threadIdx.x] = LzStep{-S.gamma, anw, S.rr};
            S.gamma_prev = S.gamma;
            S.alpha = anw;
            S.c = c_new;
            S.pp = pp_new;
            S.rr = rr_new;
            S.k = S.k + 1;
            s_anw[threadIdx.x] = anw;
            s_rn[threadIdx.x] = sqrt(rr_new);
        }
        if (threadIdx.x == 0) *counter = 0u;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kTB * ns; q += kBlock) {
        const int tt = q / ns, sh = q - tt * ns;
        SolveState &S = st[tt];
        ShiftState &h = S.sh[sh];
        if (S.done || !h.active) continue;
        const double ratio = h.ratio, zn = h.z * ratio;
        h.a = s_anw[tt] * ratio * ratio;
        h.z_prev = h.z;
        h.z = zn;
        h.iters = S.k;
        const double rz = fabs(zn) * s_rn[tt];
        h.res = rz * S.inv_bnorm;
        if (!S.fixed && (rz < S.tol * S.bnorm || !(fabs(zn) > 0.0))) h.active = 0;
    }
    __syncthreads();
    if (threadIdx.x < kTB) {
        SolveState &S = st[threadIdx.x];
        if (!S.done) {
            int na = 0;
            for (int sh = 0; sh < ns; ++sh) na += S.sh[sh].active;
            S.nactive = na;
            if (na == 0 || S.k >= S.limit || S.status != SDA_OK || s_exact[threadIdx.x]) {
                S.done = 1;
                S.alpha = 0.0;   // a stopped target's vectors stay put (gamma 0, p = r)
                S.gamma = 0.0;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1;
        for (int q = 0; q < kTB; ++q) all &= st[q].done;
        ctl->k = ctl->k + 1;
        ctl->done = all;
    }
}

// ---------------------------------------------------------------------------
// stored-basis (Lanczos) form of the shifted solutions (Sec. 3.2.1)
// ---------------------------------------------------------------------------
// Per (lane t, shift s): the solution of the shifted system in the Krylov basis
// of the lane's run.  With the CG scalars a_j (step), b_j (alpha_{j+1}) and
// ||r_j||, the Lanczos vectors are v_j = (-1)^j r_j / ||r_j|| and the base
// system's tridiagonal T has T_jj = 1/a_j + b_{j-1}/a_{j-1} and
// T_{j,j-1} = T_{j-1,j} = sqrt(b_{j-1}) / a_{j-1}.  The shift solves
// (T_K + delta_s I) y = ||r_0|| e_1 with K its stop iteration (Thomas
// algorithm, FP64; T_K + delta I is SPD), so w_s = V_K y; the coefficients of
// the raw residuals go to coef[t][s][j] = y_j (-1)^j / ||r_j|| (0 for j >= K).
// `cp` is scratch of coef's size.
__global__ void kb_lz_solve(int nl, int ns, int kmax, const LzStep *__restrict__ lz, const SolveState *st,
                            double *__restrict__ coef, double *__restrict__ cp) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nl * ns) return;
    const int t = q / ns, s = q - t * ns;
    const SolveState &S = st[t];
    double *y = coef + (int64_t)q * kmax, *c = cp + (int64_t)q * kmax;
    const int K = S.status == SDA_OK ? min(S.sh[s].iters, kmax) : 0;
    for (int j = K; j < kmax; ++j) y[j] = 0.0;
    if (K <= 0) return;
    const double delta = S.sh[s].delta;
    double pa = 1.0, pb = 0.0, cprev = 0.0, dprev = 0.0;   // a_{j-1}, b_{j-1}, forward-sweep values
    for (int j = 0; j < K; ++j) {
        const LzStep z = lz[(int64_t)j * kTB + t];
        const double sub = j > 0 ? sqrt(pb) / pa : 0.0;
        const double diag = 1.0 / z.a + (j > 0 ? pb / pa : 0.0) + delta;
        const double m = diag - sub * cprev;
        cprev = j + 1 < K ? (sqrt(z.b) / z.a) / m : 0.0;
        dprev = ((j == 0 ? sqrt(z.rr) : 0.0) - sub * dprev) / m;
        c[j] = cprev;
        y[j] = dprev;
        pa = z.a;
        pb = z.b;
    }
    for (int j = K - 2; j >= 0; --j) y[j] -= c[j] * y[j + 1];
    for (int j = 0; j < K; ++j) y[j] *= ((j & 1) ? -1.0 : 1.0) / sqrt(lz[(int64_t)j * kTB + t].rr);
}

// W = V Y of every lane: wall[l][s][j] = sum_k coef[l][s][k] r_k[j][l] over the
// basis slots k < kmax (FP64 out, permuted order).  One thread per (feature,
// lane) element and EPT features; the shifts in passes of kGemmSG accumulators
// per element (FMA in the vector type, coefficients rounded to it); a k-chunk of
// coefficients staged in shared memory; the outputs leave through a transposed
// tile so that each lane's row of features is written contiguously.
constexpr int kGemmSG = 16;
constexpr int kGemmKC = 16;
template <class FT, int EPT>
__global__ void __launch_bounds__(kBlock) kb_basis_gemm(int64_t d, int64_t ldw, int nl, int ns, int kmax,
                                                       FT *const *__restrict__ tab, int per_chunk,
                                                       const double *__restrict__ coef, double *__restrict__ wall) {
    constexpr int FR = kBlock / kTB;         // features per row of the block tile
    constexpr int FPB = FR * EPT;            // features per block tile
    __shared__ FT cs[kGemmKC][kGemmSG][kTB];
    __shared__ double tile[kTB][FPB + 1];
    const int l = threadIdx.x % kTB, f = threadIdx.x / kTB;
    const int64_t ntiles = (d + FPB - 1) / FPB;
    for (int64_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const int64_t j0 = ti * FPB;
        for (int s0 = 0; s0 < ns; s0 += kGemmSG) {
            FT acc[EPT][kGemmSG];
#pragma unroll
            for (int u = 0; u < EPT; ++u)
#pragma unroll
                for (int g = 0; g < kGemmSG; ++g) acc[u][g] = (FT)0;
            for (int k0 = 0; k0 < kmax; k0 += kGemmKC) {
                __syncthreads();
                for (int q = threadIdx.x; q < kGemmKC * kGemmSG * kTB; q += kBlock) {
                    const int kk = q / (kGemmSG * kTB), g = (q / kTB) % kGemmSG, ll = q % kTB;
                    const int k = k0 + kk, sh = s0 + g;
                    cs[kk][g][ll] = (k < kmax && sh < ns && ll < nl) ? (FT)coef[((int64_t)ll * ns + sh) * kmax + k]
                                                                     : (FT)0;
                }
                __syncthreads();
                const int kn = min(kGemmKC, kmax - k0);
                for (int kk = 0; kk < kn; ++kk) {
                    const int k = k0 + kk;
                    const FT *slot = tab[k / per_chunk] + (int64_t)(k % per_chunk) * ldw * kTB;
                    FT r[EPT];
#pragma unroll
                    for (int u = 0; u < EPT; ++u) {
                        const int64_t j = j0 + f + u * FR;
                        r[u] = j < d ? slot[j * kTB + l] : (FT)0;
                    }
#pragma unroll
                    for (int g = 0; g < kGemmSG; ++g) {
                        const FT cg = cs[kk][g][l];
#pragma unroll
                        for (int u = 0; u < EPT; ++u) acc[u][g] = fma(cg, r[u], acc[u][g]);
                    }
                }
            }
#pragma unroll
            for (int g = 0; g < kGemmSG; ++g) {
                if (s0 + g >= ns) break;
                __syncthreads();
#pragma unroll
                for (int u = 0; u < EPT; ++u) tile[l][f + u * FR] = (double)acc[u][g];
                __syncthreads();
                for (int q = threadIdx.x; q < kTB * FPB; q += kBlock) {
                    const int ll = q / FPB, jj = q % FPB;
                    const int64_t j = j0 + jj;
                    if (ll < nl && j < d) wall[((int64_t)ll * ns + s0 + g) * d + j] = tile[ll][jj];
                }
            }
        }
    }
}

// Condition of the device-driven iteration loop: keep iterating while some lane
// of the batch is still running (and the iteration cap is not passed)
__global__ void kb_loop_cond(BatchCtl *ctl, int limit, int nb_iters, cudaGraphConditionalHandle h) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int bodies = ++ctl->bodies;   // at most (limit + nb_iters) / nb_iters bodies, whatever the state
        const bool more = !ctl->done && ctl->k <= limit && (int64_t)bodies * nb_iters <= (int64_t)limit + nb_iters;
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
}

// the source vector of every lane of a [len][kTB] block (NULL: a zero lane)
template <class S>
struct LaneSrc {
    const S *p[kTB];
};

// dst[i][l] = src.p[l][i] (converted) for i < len, 0 for len <= i < len_dst or a
// NULL lane: a whole [len_dst][kTB] block in one pass
template <class S, class T>
__global__ void __launch_bounds__(kBlock) kb_put_lanes(int64_t len, int64_t len_dst, LaneSrc<S> src, T *__restrict__ dst) {
    const int64_t m = len_dst * kTB;
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m; e += (int64_t)gridDim.x * kBlock) {
        const int64_t i = e / kTB;
        const S *q = src.p[e - i * kTB];
        dst[e] = (q && i < len) ? (T)q[i] : (T)0;
    }
}
// every lane of a [len][kTB] block from one plain vector
template <class T>
__global__ void kb_rep(int64_t len, const T *__restrict__ src, T *__restrict__ dst) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len * kTB; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = src[e / kTB];
}
// w[s][j] (FP64, permuted order) of target t from W[s][j][t]
template <class FT>
__global__ void kb_take_w(int64_t d, int64_t ldw, int ns, const FT *__restrict__ W, int t, double *__restrict__ out) {
    const int64_t m = (int64_t)ns * d;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sh = i / d, j = i - sh * d;
        out[i] = (double)W[(sh * ldw + j) * kTB + t];
    }
}
// w[j] += W[0][j][t] in FP64 (a refinement correction added to its solution)
template <class FT>
__global__ void kb_add_lane(int64_t d, const FT *__restrict__ W, int t, double *__restrict__ w) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < d; j += (int64_t)gridDim.x * blockDim.x)
        w[j] += (double)W[j * kTB + t];
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
static int grid_for(const void *kernel, int sms, size_t dyn_smem = 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kBlock, dyn_smem) != cudaSuccess || nb <= 0) {
        (void)cudaGetLastError();
        nb = 1;
    }
    return std::min(nb, kMaxBlocksPerSm) * sms;
}
static int grid_elems_b(int64_t m, int sms) {
    const int64_t g = (m + kBlock - 1) / kBlock;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)sms * 16));
}
template <class S, class T>
static int put_lanes(int64_t len, int64_t len_dst, const LaneSrc<S> &src, T *dst, int sms, cudaStream_t s) {
    kb_put_lanes<S, T><<<grid_elems_b(len_dst * kTB, sms), kBlock, 0, s>>>(len, len_dst, src, dst);
    SDA_LAUNCHED();
    return SDA_OK;
}

template <class FT>
struct BView {
    typename RPair<FT>::T *pairs;
    typename CompSum<FT>::Part *s;
    FT *ut, *v, *W, *P;
    BatchCoef<FT> *coef;
    FT *p;   // p_k [ldw][kTB]
};

template <class FT>
static BView<FT> bview(BatchWs &b) {
    using Part = typename CompSum<FT>::Part;
    char *base = b.vec.p;
    auto *pairs = (typename RPair<FT>::T *)base;
    base += 2 * b.ldw * kTB * sizeof(typename RPair<FT>::T);
    auto *s = (Part *)base;
    base += b.ldw * kTB * sizeof(Part);
    FT *ut = (FT *)base, *v = ut + b.n8 * kTB;
    FT *W = (FT *)b.shift.p, *P = W ? W + (int64_t)b.shift_ns * b.ldw * kTB : nullptr;
    return BView<FT>{pairs, s, ut, v, W, P, (BatchCoef<FT> *)b.coef.p, v + b.n8 * kTB};
}

// the captured graphs hold buffer addresses: dropped whenever a buffer is reallocated
static void drop_graphs(BatchWs &b) {
    if (b.loop) cudaGraphExecDestroy(b.loop);
    b.loop = nullptr;
    b.loop_iters = 0;
}

template <class FT>
static int ensure_batch_ws(sda_operator *op, BatchWs *&slot, int ns) {
    if (!slot) slot = new BatchWs();
    BatchWs &b = *slot;
    using Part = typename CompSum<FT>::Part;
    const int fp64 = std::is_same<FT, double>::value;
    const int64_t ldw = (op->d + 7) / 8 * 8, n8 = (op->n + 7) / 8 * 8;
    if (b.fp64 == fp64 && b.d == op->d && b.n == op->n && b.ns >= ns) return SDA_OK;
    drop_graphs(b);
    SDA_TRY(b.vec.alloc((size_t)(2 * ldw * kTB * sizeof(typename RPair<FT>::T) + ldw * kTB * sizeof(Part) +
                                 2 * n8 * kTB * sizeof(FT) + ldw * kTB * sizeof(FT))));
    b.shift.release();
    b.shift_ns = 0;
    b.bchunks.clear();
    b.btab.release();
    b.btab_cap = 0;
    SDA_TRY(b.b.alloc((size_t)(ldw * kTB)));
    SDA_TRY(b.mu64.alloc((size_t)(ldw * kTB)));
    SDA_TRY(b.mu32.alloc((size_t)(ldw * kTB)));
    SDA_TRY(b.ylab.alloc((size_t)(n8 * kTB)));
    SDA_TRY(b.st.alloc(kTB));
    SDA_TRY(b.ctl.alloc(1));
    SDA_TRY(b.coef.alloc((size_t)kMaxShifts * kTB * sizeof(BatchCoef<FT>)));
    SDA_TRY(b.part.alloc((size_t)kMaxBlocksPerSm * op->sm_count * kTB * 5));   // phase 2: 2 per target, 3b: 3
    SDA_TRY(b.cnt.alloc(4));
    SDA_CUDA(cudaMemset(b.cnt.p, 0, b.cnt.bytes()));
    SDA_TRY(b.slots.alloc((size_t)std::max(std::max(op->col.nslots, op->col_tail.nslots), 1) * kTB * 2));
    SDA_TRY(b.lcount.alloc((size_t)std::max(std::max(op->col.nsplits, op->col_tail.nsplits), 1)));
    SDA_TRY(b.hparts.alloc((size_t)std::max<int64_t>(1, (int64_t)op->hb.nranges * op->hb.nseg * kTB)));
    if (fp64) {
        SDA_TRY(b.fx_planes.alloc((size_t)(std::max(ldw, n8) * kTB)));
        SDA_TRY(b.fx_amax.alloc(kTB));
        SDA_TRY(b.fx_k.alloc(kTB));
    }
    b.grid_fx1 = b.grid_fx3 = b.grid_fx_head = 0;
    SDA_CUDA(cudaMemset(b.lcount.p, 0, b.lcount.bytes()));
    SDA_TRY(b.sig.alloc(kTB));
    SDA_TRY(b.r2.alloc(kTB));
    if (!b.h_st) SDA_CUDA(cudaMallocHost(&b.h_st, sizeof(SolveState) * kTB));
    if (!b.h_ctl) SDA_CUDA(cudaMallocHost(&b.h_ctl, sizeof(BatchCtl)));
    b.fp64 = fp64;
    b.d = op->d;
    b.n = op->n;
    b.ldw = ldw;
    b.n8 = n8;
    b.ns = ns;
    b.grid = 0;
    b.tuned = false;
    return SDA_OK;
}

template <class FT>
static int ensure_batch(sda_operator *op, int ns) {
    return ensure_batch_ws<FT>(op, op->bws, ns);
}

// W, P of ns shifts for the recurrence form (grown on demand; a new buffer
// invalidates the captured graph, which holds its address)
template <class FT>
static int ensure_shift(BatchWs &b, int ns) {
    if (b.shift_ns >= ns) return SDA_OK;
    drop_graphs(b);
    SDA_TRY(b.shift.alloc((size_t)(2 * (int64_t)ns * b.ldw * kTB * sizeof(FT))));
    b.shift_ns = ns;
    return SDA_OK;
}

constexpr int kBasisChunk = 64;   // basis slots per allocated chunk

// Basis slots [0, nslots) allocated (whole chunks) and listed in the device table
// of `cap` entries; the table is (re)allocated for `cap` chunks when smaller.
template <class FT>
static int ensure_basis(BatchWs &b, int64_t nslots, int cap, cudaStream_t s) {
    if (b.btab_cap < cap) {
        drop_graphs(b);
        SDA_TRY(b.btab.alloc((size_t)cap * sizeof(FT *)));
        b.btab_cap = cap;
        std::vector<FT *> h(b.bchunks.size());
        for (size_t i = 0; i < h.size(); ++i) h[i] = (FT *)b.bchunks[i]->p;
        if (!h.empty()) {
            SDA_CUDA(cudaMemcpyAsync(b.btab.p, h.data(), h.size() * sizeof(FT *), cudaMemcpyHostToDevice, s));
            SDA_CUDA(cudaStreamSynchronize(s));
        }
    }
    const int64_t need = (nslots + kBasisChunk - 1) / kBasisChunk;
    if (need > b.btab_cap) return fail(SDA_ERR_INVALID_ARG, "basis table too small");
    while ((int64_t)b.bchunks.size() < need) {
        std::unique_ptr<DevBuf<char>> c(new DevBuf<char>());
        SDA_TRY(c->alloc((size_t)kBasisChunk * b.ldw * kTB * sizeof(FT)));
        FT *ptr = (FT *)c->p;
        SDA_CUDA(cudaMemcpyAsync((FT **)b.btab.p + b.bchunks.size(), &ptr, sizeof(FT *), cudaMemcpyHostToDevice, s));
        SDA_CUDA(cudaStreamSynchronize(s));   // `ptr` lives on this stack frame
        b.bchunks.push_back(std::move(c));
    }
    return SDA_OK;
}

// S = X^T V for the kTB vectors of a workspace: the head columns from range
// slices of V in shared memory (kb_head3a, then the fixed-order sum over the
// ranges), the other columns with the tile pass over the CSC (kb_phase3a)
template <class VT, class FT>
static int colpass_b(sda_operator *op, BatchWs &b, const FT *v, typename CompSum<FT>::Part *out, int grid_tail,
                     cudaStream_t s) {
    using Part = typename CompSum<FT>::Part;
    // head_items 0 (the autotuner's choice where the tile pass alone is faster): every
    // column through the tile pass over the operator's full column schedule
    const int64_t H = b.head_items > 0 ? op->hb.nseg : 0;
    const ColSchedule &cs = H > 0 ? op->col_tail : op->col;
    if (H > 0) {
        const size_t smem = (size_t)kHeadRows * kTB * sizeof(FT);
        if (!b.head_ready) {
            SDA_CUDA(cudaFuncSetAttribute((const void *)kb_head3a<BVT<VT>, FT>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            int nb = 0;
            SDA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)kb_head3a<BVT<VT>, FT>, kBlock,
                                                                   smem));
            b.grid_head = std::max(1, std::min(nb, kMaxBlocksPerSm)) * op->sm_count;
            b.head_ready = true;
        }
        // slices of the head columns per range: at least four items per resident block
        const int nr = op->hb.nranges;
        const int nsplit =
            (int)std::max<int64_t>(1, std::min<int64_t>(H / 64, ((int64_t)b.head_items * b.grid_head + nr - 1) / nr));
        kb_head3a<BVT<VT>, FT><<<std::min(b.grid_head, nr * nsplit), kBlock, smem, s>>>(
            op->n, nr, (int)H, nsplit, op->hb.cp.p, op->hb.idx.p, (const BVT<VT> *)op->hb.val.p, v,
            (Part *)b.hparts.p, b.ctl.p);
        SDA_LAUNCHED();
        const int64_t m = H * kTB;
        kb_head_reduce<FT><<<(int)std::min<int64_t>((m + 31) / 32, (int64_t)op->sm_count * 8), kBlock, 0, s>>>(
            op->hb.nranges, m, (const Part *)b.hparts.p, out, b.ctl.p);
        SDA_LAUNCHED();
    }
    kb_phase3a<VT, FT><<<grid_tail, kBlock, 0, s>>>(cs.tiles.p, cs.ntiles, op->x_cp.p + H, op->x_row.p,
                                                    (const VT *)op->x_val_c.p, v, out + H * kTB, (Part *)b.slots.p,
                                                    b.lcount.p, cs.splits.p, b.ctl.p);
    SDA_LAUNCHED();
    return SDA_OK;
}

// U = X P - 1 c^T for the kTB vectors of a workspace (row pass over the quad-padded rows)
template <class VT, class FT>
static int rowpass_b(sda_operator *op, BatchWs &b, const FT *p, FT *ut, int grid, cudaStream_t s) {
    kb_phase1<BVT<VT>, FT><<<grid, kBlock, 0, s>>>(op->n, b.ldw, op->xr_rp.p, op->xr_col.p,
                                                  (const BVT<VT> *)op->xr_val.p, p, ut, b.st.p, b.ctl.p);
    SDA_LAUNCHED();
    return SDA_OK;
}

// launches of colpass_b
static int colpass_launches(const sda_operator *op, const BatchWs &b) {
    return op->hb.nseg > 0 && b.head_items > 0 ? 3 : 1;
}

// `ev` (profile mode): a start and an end event around each of the four kernels
template <class VT, class FT>
static int batch_iteration(sda_operator *op, int ns, bool basis, cudaStream_t s, cudaEvent_t *ev = nullptr) {
    BatchWs &b = *op->bws;
    BView<FT> bv = bview<FT>(b);
    const BasisView<FT> bvw{basis ? (FT *const *)b.btab.p : nullptr, kBasisChunk, basis ? b.lz.p : nullptr};
    const FT *sv = std::is_same<FT, double>::value ? (const FT *)op->s_val64.p : (const FT *)op->s_val32.p;
    const FT *dg = std::is_same<FT, double>::value ? (const FT *)op->deg64.p : (const FT *)op->deg32.p;
    const int P = kMaxBlocksPerSm * op->sm_count;
    if (ev) SDA_CUDA(cudaEventRecord(ev[0], s));
    kb_formp<FT><<<b.grid, kBlock, 0, s>>>(op->d, b.ldw, bv.pairs, bv.p, b.st.p, b.ctl.p);
    SDA_LAUNCHED();
    SDA_TRY((rowpass_b<VT, FT>(op, b, bv.p, bv.ut, b.grid1, s)));

    if (ev) SDA_CUDA(cudaEventRecord(ev[1], s));
    if (ev) SDA_CUDA(cudaEventRecord(ev[2], s));
    kb_phase2<FT><<<b.grid2, kBlock, 0, s>>>(op->n, op->s_rp.p, op->s_col.p, sv, bv.ut, dg, b.ylab.p, bv.v, b.st.p,
                                            b.ctl.p, bv.coef, ns, b.part.p, b.cnt.p + 0);
    SDA_LAUNCHED();

    using Part = typename CompSum<FT>::Part;
    if (ev) SDA_CUDA(cudaEventRecord(ev[3], s));
    if (ev) SDA_CUDA(cudaEventRecord(ev[4], s));
    SDA_TRY((colpass_b<VT, FT>(op, b, bv.v, bv.s, b.grid3a, s)));

    if (ev) SDA_CUDA(cudaEventRecord(ev[5], s));
    if (ev) SDA_CUDA(cudaEventRecord(ev[6], s));
    kb_phase3b<FT><<<b.grid, kBlock, (size_t)ns * kTB * sizeof(BatchCoef<FT>), s>>>(
        op->d, b.ldw, ns, bv.s, bv.pairs, basis ? nullptr : bv.W, basis ? nullptr : bv.P, b.st.p, b.ctl.p, bv.coef,
        b.mu32.p, b.mu64.p, b.part.p + (int64_t)P * kTB * 2, b.cnt.p + 1, bvw);
    SDA_LAUNCHED();
    if (ev) SDA_CUDA(cudaEventRecord(ev[7], s));

    return SDA_OK;
}

// nb_iters iterations launched from the host: with events around every phase
// (profile mode), else plain launches (graphs off)
template <class VT, class FT>
static int batch_run(sda_operator *op, int ns, bool basis, int nb_iters, bool profile, cudaStream_t s) {
    if (profile) {
        std::vector<cudaEvent_t> &pe = op->ws.prof_ev;
        while (pe.size() < (size_t)nb_iters * 8) {
            cudaEvent_t e;
            SDA_CUDA(cudaEventCreate(&e));
            pe.push_back(e);
        }
        for (int i = 0; i < nb_iters; ++i) SDA_TRY((batch_iteration<VT, FT>(op, ns, basis, s, pe.data() + 8 * i)));
        SDA_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < nb_iters; ++i)
            for (int ph = 0; ph < 4; ++ph) {
                float ms = 0.f;
                SDA_CUDA(cudaEventElapsedTime(&ms, pe[8 * i + 2 * ph], pe[8 * i + 2 * ph + 1]));
                op->stats.ms[1 + ph] += ms;
            }
        for (int ph = 1; ph <= 4; ++ph) op->stats.launches[ph] += nb_iters;
        return SDA_OK;
    }
    for (int i = 0; i < nb_iters; ++i) SDA_TRY((batch_iteration<VT, FT>(op, ns, basis, s)));
    for (int ph = 1; ph <= 4; ++ph) op->stats.launches[ph] += nb_iters;
    return SDA_OK;
}

// The whole run of a batch as one graph launch: a WHILE node whose body is
// nb_iters iterations and kb_loop_cond, so the device decides when the batch
// is done (no host round trip between iterations).  Returns the bodies run.
template <class VT, class FT>
static int batch_loop(sda_operator *op, int ns, bool basis, int nb_iters, int limit, cudaStream_t s) {
    BatchWs &b = *op->bws;
    if (!b.loop || b.loop_iters != nb_iters || b.loop_ns != ns || b.loop_basis != (int)basis || b.loop_limit != limit) {
        if (b.loop) cudaGraphExecDestroy(b.loop);
        b.loop = nullptr;
        if (!b.cap_stream) SDA_CUDA(cudaStreamCreateWithFlags(&b.cap_stream, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        SDA_CUDA(cudaGraphCreate(&g, 0));
        cudaGraphConditionalHandle h;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
        cudaGraphNodeParams np = {};
        cudaGraphNode_t node = nullptr;
        if (e == cudaSuccess) {
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
        }
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_fail(e, "conditional graph node", __FILE__, __LINE__);
        }
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(b.cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_fail(e, "cudaStreamBeginCaptureToGraph", __FILE__, __LINE__);
        }
        set_capturing(true);
        int rc = SDA_OK;
        for (int i = 0; i < nb_iters && rc == SDA_OK; ++i) rc = batch_iteration<VT, FT>(op, ns, basis, b.cap_stream);
        if (rc == SDA_OK) {
            kb_loop_cond<<<1, 32, 0, b.cap_stream>>>(b.ctl.p, limit, nb_iters, h);
            if (cudaGetLastError() != cudaSuccess) rc = fail(SDA_ERR_CUDA, "loop condition launch failed");
        }
        set_capturing(false);
        cudaGraph_t cap = nullptr;
        e = cudaStreamEndCapture(b.cap_stream, &cap);
        if (rc == SDA_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b.loop, g, 0);
        cudaGraphDestroy(g);
        if (rc != SDA_OK) return rc;
        if (e != cudaSuccess) return cuda_fail(e, "device-driven loop graph", __FILE__, __LINE__);
        b.loop_iters = nb_iters;
        b.loop_ns = ns;
        b.loop_basis = (int)basis;
        b.loop_limit = limit;
    }
    SDA_CUDA(cudaGraphLaunch(b.loop, s));
    return SDA_OK;
}

// ---------------------------------------------------------------------------
// autotuner of the batched sparse passes
// ---------------------------------------------------------------------------
// Schedules picked per problem shape (rows, features, nonzeros of X and S, value
// type, vector type, SMs) and kept for the process: resident blocks per SM of the
// row pass, the Laplacian pass and the tail column pass, and work items per
// resident block of the head column pass.
using TuneKey = std::tuple<int64_t, int64_t, int64_t, int64_t, int, int, int>;
struct TuneVal {
    int bpsm1, bpsm2, bpsm3, head_items;
};
static std::map<TuneKey, TuneVal> g_tuned;
static std::mutex g_tune_mu;

// device time of `launch` (ms, the best of three runs of two launches)
template <class F>
static int time_launch(cudaStream_t s, F &&launch, float *best) {
    cudaEvent_t e0, e1;
    SDA_CUDA(cudaEventCreate(&e0));
    SDA_CUDA(cudaEventCreate(&e1));
    *best = 1e30f;
    int rc = SDA_OK;
    for (int rep = 0; rep < 3 && rc == SDA_OK; ++rep) {
        cudaEventRecord(e0, s);
        rc = launch();
        if (rc == SDA_OK) rc = launch();
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(SDA_ERR_CUDA, "autotuner timing failed");
        float ms = 0.f;
        if (rc == SDA_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) *best = std::min(*best, ms / 2);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

// Picks the schedule of op's batched sparse passes for vector type FT (once per
// shape in the process) and sets b's grids.  The passes run on the workspace's
// current vectors; the solve state they touch is reset by the run that follows.
template <class VT, class FT>
static int autotune(sda_operator *op, BatchWs &b, cudaStream_t s) {
    const TuneKey key{op->n, op->d, op->nnz, op->s_nnz, (int)op->compute, (int)sizeof(FT), op->sm_count};
    TuneVal tv{0, 0, 0, 0};
    bool have = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            tv = it->second;
            have = true;
        }
    }
    const int sms = op->sm_count;
    if (!have) {
        BatchCtl hc{};
        hc.bb = BatchBounds{op->n, op->d, b.ldw, b.n8, op->nnz, op->s_nnz, op->col.ntiles,
                            std::max(op->col.nslots, op->col_tail.nslots), std::max(op->col.nsplits, op->col_tail.nsplits),
                            (int64_t)b.part.n, (int64_t)(op->xr_col.n / 4)};
        *b.h_ctl = hc;
        SDA_CUDA(cudaMemcpyAsync(b.ctl.p, b.h_ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, s));
        SDA_CUDA(cudaMemsetAsync(b.vec.p, 0, b.vec.bytes(), s));
        BView<FT> bv = bview<FT>(b);
        const FT *sv = std::is_same<FT, double>::value ? (const FT *)op->s_val64.p : (const FT *)op->s_val32.p;
        const FT *dg = std::is_same<FT, double>::value ? (const FT *)op->deg64.p : (const FT *)op->deg32.p;
        const int cand[4] = {2, 3, 4, 6};
        const int m1 = b.grid1 / sms, m2 = b.grid2 / sms, m3 = b.grid3a / sms;   // occupancy caps
        float best1 = 1e30f, best2 = 1e30f, best3 = 1e30f, t = 0.f;
        for (int c : cand) {
            if (c <= m1) {
                SDA_TRY(time_launch(s, [&] { return rowpass_b<VT, FT>(op, b, bv.p, bv.ut, c * sms, s); }, &t));
                if (t < best1) best1 = t, tv.bpsm1 = c;
            }
            if (c <= m2) {
                SDA_TRY(time_launch(s, [&]() -> int {
                    kb_phase2<FT><<<c * sms, kBlock, 0, s>>>(op->n, op->s_rp.p, op->s_col.p, sv, bv.ut, dg, b.ylab.p,
                                                             bv.v, b.st.p, b.ctl.p, bv.coef, 0, b.part.p, b.cnt.p + 0);
                    SDA_LAUNCHED();
                    return SDA_OK;
                }, &t));
                if (t < best2) best2 = t, tv.bpsm2 = c;
            }
            if (c <= m3) {
                SDA_TRY(time_launch(s, [&]() -> int {
                    const int64_t H = op->hb.nseg;
                    using Part = typename CompSum<FT>::Part;
                    kb_phase3a<VT, FT><<<c * sms, kBlock, 0, s>>>(op->col_tail.tiles.p, op->col_tail.ntiles,
                                                                 op->x_cp.p + H, op->x_row.p, (const VT *)op->x_val_c.p,
                                                                 bv.v, bv.s + H * kTB, (Part *)b.slots.p, b.lcount.p,
                                                                 op->col_tail.splits.p, b.ctl.p);
                    SDA_LAUNCHED();
                    return SDA_OK;
                }, &t));
                if (t < best3) best3 = t, tv.bpsm3 = c;
            }
        }
        tv.head_items = 4;
        if (op->hb.nseg > 0) {
            // head columns from shared-memory range slices (items per resident block
            // 1..8), or no head pass at all: every column through the tile pass
            float besth = 1e30f;
            for (int items : {1, 2, 4, 8, 0}) {
                b.head_items = items;
                SDA_TRY(time_launch(s, [&] { return colpass_b<VT, FT>(op, b, bv.v, bv.s, b.grid3a, s); }, &t));
                if (t < besth) besth = t, tv.head_items = items;
            }
        }
        if (tv.bpsm1 == 0) tv.bpsm1 = std::max(1, m1);
        if (tv.bpsm2 == 0) tv.bpsm2 = std::max(1, m2);
        if (tv.bpsm3 == 0) tv.bpsm3 = std::max(1, m3);
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tuned[key] = tv;
    }
    b.grid1 = tv.bpsm1 * sms;
    b.grid2 = tv.bpsm2 * sms;
    b.grid3a = tv.bpsm3 * sms;
    b.head_items = tv.head_items;
    b.tuned = true;
    op->tuned[0] = tv.bpsm1;
    op->tuned[1] = tv.bpsm2;
    op->tuned[2] = tv.bpsm3;
    op->tuned[3] = tv.head_items > 0 ? tv.head_items : -1;
    return SDA_OK;
}

// One lane of a batched shifted-CG run: the operator target whose labels and
// mu_l it uses, its right-hand side (device, permuted order), the base shift
// sigma0 of its Krylov run and its relative stop tolerance.
struct BatchLane {
    int t;
    const double *b;
    double sigma0;
    double tol;
};

// Shifted CG (Algorithm 3) on nl <= kTB lanes in lockstep: lane l solves
// (B_{t_l} + (sigma0_l + delta_s) I) w = b_l for the ns relative shifts
// delta_s (shared by the lanes).  Lanes past nl hold a zero right-hand side
// and stop at once.  Leaves every lane's W^s in the workspace ([s][j][lane])
// and the final solve states in the workspace's h_st.
template <class VT, class FT>
static int run_lanes(sda_operator *op, const BatchLane *lanes, int nl, const double *deltas, int ns, bool fixed,
                     int limit, const sda_solve_opts &o, double alpha, double omega, cudaStream_t s,
                     bool basis = false) {
    SDA_TRY(ensure_batch<FT>(op, ns));
    BatchWs &b = *op->bws;
    const int nbi = o.iter_batch > 0 ? o.iter_batch : 32;
    if (basis) {
        // slots up to the last launched iteration, CG scalars of every iteration
        const int64_t max_slots = (int64_t)limit + nbi + 1;
        SDA_TRY(ensure_basis<FT>(b, 0, (int)((max_slots + kBasisChunk - 1) / kBasisChunk), s));
        if (b.lz.n < (size_t)max_slots * kTB) SDA_TRY(b.lz.alloc((size_t)max_slots * kTB));
    } else {
        SDA_TRY(ensure_shift<FT>(b, ns));
    }
    if (!b.grid) {
        SDA_CUDA(cudaFuncSetAttribute((const void *)kb_phase3b<FT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(kMaxShifts * kTB * sizeof(BatchCoef<FT>))));
        b.grid1 = grid_for((const void *)kb_phase1<BVT<VT>, FT>, op->sm_count);
        b.grid2 = grid_for((const void *)kb_phase2<FT>, op->sm_count);
        b.grid3a = grid_for((const void *)kb_phase3a<VT, FT>, op->sm_count);
        b.grid = std::min(std::min(b.grid1, b.grid2), std::min(b.grid3a, grid_for((const void *)kb_phase3b<FT>, op->sm_count,
                                                                    kMaxShifts * kTB * sizeof(BatchCoef<FT>))));
    }
    if (!b.tuned) SDA_TRY((autotune<VT, FT>(op, b, s)));
    const int64_t d = op->d, n = op->n;
    {
        LaneSrc<double> rb{}, mu{};
        LaneSrc<int8_t> yl{};
        for (int i = 0; i < nl; ++i) {
            const int t = lanes[i].t;
            rb.p[i] = lanes[i].b;
            mu.p[i] = op->mu.p + (int64_t)t * d;
            yl.p[i] = op->labels.p + (int64_t)t * n;
        }
        SDA_TRY(put_lanes(d, b.ldw, rb, b.b.p, op->sm_count, s));
        SDA_TRY(put_lanes(d, b.ldw, mu, b.mu64.p, op->sm_count, s));
        SDA_TRY(put_lanes(d, b.ldw, mu, b.mu32.p, op->sm_count, s));
        SDA_TRY(put_lanes(n, b.n8, yl, b.ylab.p, op->sm_count, s));
    }
    SolveState *h = b.h_st;
    memset(h, 0, sizeof(SolveState) * kTB);
    for (int l = 0; l < kTB; ++l) {
        const BatchLane &ln = lanes[l < nl ? l : 0];
        h[l].sigma0 = ln.sigma0;
        h[l].omega = omega;
        h[l].alpha_l = alpha;
        h[l].tol = ln.tol;
        h[l].n_shifts = ns;
        h[l].fixed = fixed ? 1 : 0;
        h[l].limit = limit;
        for (int i = 0; i < ns; ++i) h[l].sh[i].delta = deltas[i];
    }
    SDA_CUDA(cudaMemcpyAsync(b.st.p, h, sizeof(SolveState) * kTB, cudaMemcpyHostToDevice, s));
    BView<FT> bv = bview<FT>(b);
    {
        BatchCtl hc{};
        hc.bb = BatchBounds{op->n, op->d, b.ldw, b.n8, op->nnz, op->s_nnz, op->col.ntiles,
                            std::max(op->col.nslots, op->col_tail.nslots), std::max(op->col.nsplits, op->col_tail.nsplits),
                            (int64_t)b.part.n, (int64_t)(op->xr_col.n / 4)};
        *b.h_ctl = hc;
        SDA_CUDA(cudaMemcpyAsync(b.ctl.p, b.h_ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, s));
    }
    kb_init<FT><<<b.grid, kBlock, 0, s>>>(b.ldw, ns, b.b.p, b.mu64.p, bv.pairs, basis ? nullptr : bv.W,
                                          basis ? nullptr : bv.P, b.st.p, b.ctl.p, b.part.p, b.cnt.p + 2);
    SDA_LAUNCHED();
    SDA_CUDA(cudaMemcpyAsync(b.h_ctl, b.ctl.p, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    const bool device_loop = o.use_graph && !o.profile && !b.h_ctl->done;
    if (device_loop) {
        // the device-driven loop: one graph launch runs the batch to its end
        if (basis) SDA_TRY(ensure_basis<FT>(b, (int64_t)limit + nbi + 1, b.btab_cap, s));
        SDA_TRY((batch_loop<VT, FT>(op, ns, basis, nbi, limit, s)));
        SDA_CUDA(cudaMemcpyAsync(b.h_ctl, b.ctl.p, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
        SDA_CUDA(cudaStreamSynchronize(s));
        if (b.h_ctl->err)
            return fail(SDA_ERR_INDEX, "batched solve: index check %llu failed at %llu",
                        (unsigned long long)(b.h_ctl->err >> 40), (unsigned long long)(b.h_ctl->err & 0xffffffffffull));
        const int64_t bodies = std::max<int64_t>(1, ((int64_t)b.h_ctl->k + nbi - 1) / nbi);
        note_launch(bodies * ((4 + colpass_launches(op, b)) * (int64_t)nbi + 1));
        for (int ph = 1; ph <= 4; ++ph) op->stats.launches[ph] += bodies * nbi;
    }
    int launched = device_loop ? limit + 1 : 0;   // the host-driven loop: profile mode and graphs off
    while (!b.h_ctl->done && launched <= limit) {
        if (basis) SDA_TRY(ensure_basis<FT>(b, (int64_t)launched + nbi, b.btab_cap, s));
        SDA_TRY((batch_run<VT, FT>(op, ns, basis, nbi, o.profile != 0, s)));
        launched += nbi;
        SDA_CUDA(cudaMemcpyAsync(b.h_ctl, b.ctl.p, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
        SDA_CUDA(cudaStreamSynchronize(s));
        if (b.h_ctl->err)
            return fail(SDA_ERR_INDEX, "batched solve: index check %llu failed at %llu",
                        (unsigned long long)(b.h_ctl->err >> 40), (unsigned long long)(b.h_ctl->err & 0xffffffffffull));
    }
    SDA_CUDA(cudaMemcpyAsync(h, b.st.p, sizeof(SolveState) * kTB, cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    int bk = 0;
    for (int l = 0; l < nl; ++l) bk = std::max(bk, h[l].k);
    op->stats.iterations += bk;   // iterations of the run (its slowest lane)
    return SDA_OK;
}

// Outcome of a batched run of lanes, per (lane, shift) pair [lane][shift]: the
// final solve states of the lanes, FP64 true residuals (-1: not computed) and
// refinement statuses.
struct LaneOutcome {
    std::vector<SolveState> fin;
    std::vector<double> tres, bn;
    std::vector<int> pst;
};

// Lanes l < nl (<= kTB) share one shifted-CG run of the ns relative shifts
// `deltas`; pair (l, s) solves (B_{t_l} + pshift[l ns + s] I) w = b_l (the run
// uses sigma0_l + delta_s for it).  Leaves the FP64 solutions in the
// workspace's wall ([l][s][D], permuted order).  Then the FP64 true residual
// of every pair and, with refine_rounds > 0, per-pair refinement: while a
// pair's FP64 true residual exceeds refine_tol, its correction
// (B_t + beta I) c = b_t - (B_t + beta I) w is solved in the iteration's
// precision and added in FP64; the corrections of up to kTB pairs (of any
// lanes and shifts, grouped by shift value) run as the lanes of one batched run.
template <class VT, class FT>
static int solve_lanes(sda_operator *op, const BatchLane *lanes, int nl, const double *deltas, const double *pshift,
                       int ns, const sda_solve_opts &o, double alpha, double omega, cudaStream_t s, LaneOutcome &out) {
    const int64_t d = op->d;
    const bool fixed = o.fixed_iters > 0;
    const int limit = fixed ? o.fixed_iters : o.max_iter;
    bool basis = o.shift_form == SDA_SHIFTS_BASIS;
    if (o.shift_form == SDA_SHIFTS_AUTO && ns > 1) {
        // the stored basis when its worst case fits 40 % of the free memory (chunks held count as free)
        size_t fr = 0, tot = 0;
        SDA_CUDA(cudaMemGetInfo(&fr, &tot));
        size_t held = 0;
        if (op->bws)
            for (const auto &c : op->bws->bchunks) held += c->bytes();
        const double need = (double)(limit + 1) * (double)((op->d + 7) / 8 * 8) * kTB * sizeof(FT);
        basis = need <= 0.4 * (double)(fr + held);
    }
    SDA_TRY((run_lanes<VT, FT>(op, lanes, nl, deltas, ns, fixed, limit, o, alpha, omega, s, basis)));
    BatchWs &b = *op->bws;
    if (op->stats.shift_form == 0) op->stats.shift_form = basis ? SDA_SHIFTS_BASIS : SDA_SHIFTS_RECURRENCE;
    out.fin.assign(b.h_st, b.h_st + kTB);   // later runs reuse h_st
    const std::vector<SolveState> &fin = out.fin;
    int kmax = 0;
    for (int i = 0; i < nl; ++i)
        for (int sh = 0; sh < ns; ++sh) {
            op->stats.shift_iterations += fin[(size_t)i].sh[sh].iters;
            kmax = std::max(kmax, fin[(size_t)i].sh[sh].iters);
        }
    const size_t wall_n = (size_t)nl * ns * d;
    if (b.wall.n < wall_n) SDA_TRY(b.wall.alloc(wall_n));
    if (basis) {
        // every shift's solution from the stored basis: its tridiagonal solve, then W = V Y
        if (op->stats.basis_slots == 0) op->stats.basis_slots = kmax;
        if (kmax > 0) {
            const size_t nc = (size_t)nl * ns * kmax;
            if (b.coefs.n < 2 * nc) SDA_TRY(b.coefs.alloc(2 * nc));
            kb_lz_solve<<<(nl * ns + 127) / 128, 128, 0, s>>>(nl, ns, kmax, b.lz.p, b.st.p, b.coefs.p,
                                                              b.coefs.p + nc);
            SDA_LAUNCHED();
            constexpr int EPT = std::is_same<FT, float>::value ? 4 : 2;
            const int64_t ntiles = (d + (kBlock / kTB) * EPT - 1) / ((kBlock / kTB) * EPT);
            const int gg = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)op->sm_count * 8));
            kb_basis_gemm<FT, EPT><<<gg, kBlock, 0, s>>>(d, b.ldw, nl, ns, kmax, (FT *const *)b.btab.p, kBasisChunk,
                                                         b.coefs.p, b.wall.p);
            SDA_LAUNCHED();
        } else {
            SDA_CUDA(cudaMemsetAsync(b.wall.p, 0, wall_n * sizeof(double), s));
        }
    } else {
        BView<FT> bv = bview<FT>(b);
        for (int i = 0; i < nl; ++i) {
            kb_take_w<FT><<<grid_elems_b((int64_t)ns * d, op->sm_count), kBlock, 0, s>>>(
                d, b.ldw, ns, bv.W, i, b.wall.p + (int64_t)i * ns * d);
            SDA_LAUNCHED();
        }
    }
    const int rounds = fixed ? 0 : std::max(0, o.refine_rounds);
    const double rtol = std::isnan(o.refine_tol) || o.refine_tol <= 0.0 ? o.tol : o.refine_tol;
    const bool check = o.check_residual != 0 || rounds > 0;
    std::vector<double> &tres = out.tres, &bn = out.bn;
    std::vector<int> &pst = out.pst;
    tres.assign((size_t)nl * ns, -1.0);
    bn.assign((size_t)nl, 0.0);
    pst.assign((size_t)nl * ns, SDA_OK);
    if (!check) return SDA_OK;
    {   // ||b_l|| of every lane
        DevBuf<double> bb;
        SDA_TRY(bb.alloc((size_t)nl));
        for (int i = 0; i < nl; ++i) SDA_TRY(dot_f64(op, d, lanes[i].b, lanes[i].b, bb.p + i, s));
        SDA_CUDA(cudaMemcpyAsync(bn.data(), bb.p, (size_t)nl * sizeof(double), cudaMemcpyDeviceToHost, s));
        SDA_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < nl; ++i) bn[(size_t)i] = sqrt(bn[(size_t)i]);
    }
    auto lane_of = [&](int q) {
        const int i = q / ns;
        return ResidLane{lanes[i].t, pshift[q], lanes[i].b, b.wall.p + (int64_t)q * d};
    };
    auto rel = [&](int q, double r2) {
        const double bq = bn[(size_t)(q / ns)];
        return bq > 0 ? sqrt(r2) / bq : sqrt(r2);
    };
    // FP64 true residual of every pair, kTB pairs per FP64 block pass
    for (int g0 = 0; g0 < nl * ns; g0 += kTB) {
        const int ng = std::min(kTB, nl * ns - g0);
        ResidLane rl[kTB];
        double r2[kTB];
        for (int g = 0; g < ng; ++g) rl[g] = lane_of(g0 + g);
        SDA_TRY(resid_lanes(op, rl, ng, r2, nullptr, alpha, omega, s));
        for (int g = 0; g < ng; ++g) tres[(size_t)(g0 + g)] = rel(g0 + g, r2[g]);
    }
    if (rounds > 0 && b.rbuf.n < (size_t)kTB * d) SDA_TRY(b.rbuf.alloc((size_t)kTB * d));
    for (int rd = 0; rd < rounds; ++rd) {
        // pairs still above the target, by shift value: a group's run lasts as long
        // as its smallest shift needs, so groups of equal shifts waste the least
        std::vector<int> act;
        for (int q = 0; q < nl * ns; ++q)
            if (tres[(size_t)q] > rtol && bn[(size_t)(q / ns)] > 0 && fin[(size_t)(q / ns)].status == SDA_OK &&
                pst[(size_t)q] == SDA_OK)
                act.push_back(q);
        if (act.empty()) break;
        std::stable_sort(act.begin(), act.end(), [&](int a, int c) { return pshift[a] < pshift[c]; });
        for (size_t g0 = 0; g0 < act.size(); g0 += kTB) {
            const int ng = (int)std::min<size_t>(kTB, act.size() - g0);
            ResidLane rl[kTB];
            double r2[kTB];
            BatchLane cl[kTB];
            for (int g = 0; g < ng; ++g) {
                const int q = act[g0 + g];
                rl[g] = lane_of(q);
                // relative reduction asked of the correction: to the target, but
                // not below what the iteration's precision can reach
                const double inner = std::min(0.5, std::max(rtol / tres[(size_t)q], 1e-4));
                cl[g] = BatchLane{rl[g].t, b.rbuf.p + (int64_t)g * d, rl[g].sigma, inner};
            }
            // residual vectors b - (B + beta) w in FP64, then the corrections
            SDA_TRY(resid_lanes(op, rl, ng, r2, b.rbuf.p, alpha, omega, s));
            const double zero = 0.0;
            SDA_TRY((run_lanes<VT, FT>(op, cl, ng, &zero, 1, false, o.max_iter, o, alpha, omega, s)));
            BView<FT> bv = bview<FT>(*op->bws);
            for (int g = 0; g < ng; ++g) {
                const int q = act[g0 + g];
                const SolveState &cs = op->bws->h_st[g];
                if (cs.status != SDA_OK) {
                    pst[(size_t)q] = cs.status;
                    continue;
                }
                kb_add_lane<FT><<<grid_elems_b(d, op->sm_count), kBlock, 0, s>>>(d, bv.W, g, b.wall.p + (int64_t)q * d);
                SDA_LAUNCHED();
            }
            SDA_TRY(resid_lanes(op, rl, ng, r2, nullptr, alpha, omega, s));
            for (int g = 0; g < ng; ++g) tres[(size_t)act[g0 + g]] = rel(act[g0 + g], r2[g]);
        }
    }
    return SDA_OK;
}

// One batch: targets t0 .. t0 + nt - 1 (nt <= kTB), every shift, as the lanes
// of one run (solve_lanes); solutions out in the caller's feature order.
template <class VT, class FT>
static int solve_batch(sda_operator *op, int t0, int nt, const double *const *b_perm, const double *shifts, int ns,
                       const sda_solve_opts &o, double alpha, double omega, double *w_out, sda_shift_report *rep,
                       cudaStream_t s, int *worst) {
    const int64_t d = op->d;
    const bool fixed = o.fixed_iters > 0;
    double sigma0 = shifts[0];
    for (int i = 1; i < ns; ++i) sigma0 = std::min(sigma0, shifts[i]);
    std::vector<double> deltas((size_t)ns), pshift((size_t)nt * ns);
    for (int i = 0; i < ns; ++i) deltas[(size_t)i] = shifts[i] - sigma0;
    BatchLane lanes[kTB];
    for (int i = 0; i < nt; ++i) {
        lanes[i] = BatchLane{t0 + i, b_perm[i], sigma0, o.tol};
        for (int sh = 0; sh < ns; ++sh) pshift[(size_t)i * ns + sh] = shifts[sh];
    }
    LaneOutcome out;
    SDA_TRY((solve_lanes<VT, FT>(op, lanes, nt, deltas.data(), pshift.data(), ns, o, alpha, omega, s, out)));
    BatchWs &b = *op->bws;
    for (int i = 0; i < nt && w_out; ++i) {
        double *dst = w_out + (int64_t)i * ns * d;
        const double *src = b.wall.p + (int64_t)i * ns * d;
        if (!o.out_on_device) {
            DevBuf<double> hostbuf;
            SDA_TRY(hostbuf.alloc((size_t)ns * d));
            SDA_TRY(permute_to_old(op, src, hostbuf.p, ns, s));
            SDA_CUDA(cudaMemcpyAsync(dst, hostbuf.p, (size_t)ns * d * sizeof(double), cudaMemcpyDeviceToHost, s));
            SDA_CUDA(cudaStreamSynchronize(s));
        } else {
            SDA_TRY(permute_to_old(op, src, dst, ns, s));
        }
    }
    const int rounds = fixed ? 0 : std::max(0, o.refine_rounds);
    const double rtol = std::isnan(o.refine_tol) || o.refine_tol <= 0.0 ? o.tol : o.refine_tol;
    for (int i = 0; i < nt; ++i) {
        const int t = t0 + i;
        const SolveState &S = out.fin[(size_t)i];
        if (S.status != SDA_OK) {
            *worst = S.status;
            fail(S.status, "breakdown in the batched shifted CG of target %d at iteration %d", t, S.k);
        }
        for (int sh = 0; sh < ns; ++sh) {
            const size_t q = (size_t)i * ns + sh;
            const ShiftState &hs = S.sh[sh];
            int st = SDA_OK;
            if (S.status != SDA_OK) st = S.status;
            else if (out.pst[q] != SDA_OK) st = out.pst[q];
            else if (rounds > 0) st = out.tres[q] <= rtol ? SDA_OK : SDA_NOT_CONVERGED;
            else if (!fixed && hs.active) st = SDA_NOT_CONVERGED;
            if (st == SDA_NOT_CONVERGED && *worst == SDA_OK) *worst = SDA_NOT_CONVERGED;
            if (st < 0 && *worst >= 0) *worst = st;
            if (rep) {
                sda_shift_report &r = rep[(int64_t)q];
                r.iters = hs.iters;
                r.status = st;
                r.est_residual = hs.res;
                r.true_residual = out.tres[q];
            }
        }
    }
    return SDA_OK;
}

template <class F>
static int with_vt_b(int compute, F &&f) {
    switch (compute) {
    case SDA_F64: return f((double *)nullptr);
    case SDA_F32: return f((float *)nullptr);
    case SDA_F16: return f((__half *)nullptr);
    case SDA_F8E4M3: return f((__nv_fp8_e4m3 *)nullptr);
    default: return f((Pattern *)nullptr);
    }
}

// ---------------------------------------------------------------------------
// FP64 utilities on blocks of 16 vectors: the batched kernels with FP64
// vectors, each lane one vector with the labels and mu_l of its own target.
// X and S are read once per 16 vectors.
// ---------------------------------------------------------------------------
// out[v][i] = U[i][v] for v < nv
__global__ void kb_unpack(int64_t n, int nv, const double *__restrict__ U, double *__restrict__ out) {
    const int64_t m = n * nv;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / n, i = e - v * n;
        out[e] = U[i * kTB + v];
    }
}
// st[v].c = <mu_v, P_v> (mu and P as [d][kTB] blocks)
__global__ void __launch_bounds__(kBlock) kb_dot_mu(int64_t d, const double *__restrict__ mu,
                                                   const double *__restrict__ P, SolveState *st, BatchCtl *ctl,
                                                   double *partials, unsigned *counter) {
    using Part = CompSum<double>::Part;
    __shared__ Part red[kBlock];
    CompSum<double> acc[1];
    const int64_t m = d * kTB;
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m; e += (int64_t)gridDim.x * kBlock)
        acc[0].add(mu[e] * P[e]);
    Part mine[1];
    block_tparts<1, double>(acc, mine, red);
    if (!arrive_last_t<1>(mine, reinterpret_cast<Part *>(partials), counter, ctl)) return;
    double tot[1];
    grid_tparts<1, double>(reinterpret_cast<const Part *>(partials), gridDim.x, tot, red);
    if (threadIdx.x < kTB) {
        st[threadIdx.x].c = tot[0];
        if (threadIdx.x == 0) *counter = 0u;
    }
}
// lane v: r = b_v - ((X~^T M_v X~) P_v + sig_v P_v) from S = X^T V and t_v = 1^T V_v;
// out[v] = ||r||^2; rvec[v][j] = r_j (v < nv) when rvec is not NULL
__global__ void __launch_bounds__(kBlock) kb_resid(int64_t d, int nv, const double *__restrict__ b,
                                                  const double *__restrict__ mu, const double *__restrict__ S,
                                                  const double *__restrict__ P, const double *__restrict__ sig,
                                                  const SolveState *st, BatchCtl *ctl, double *out,
                                                  double *__restrict__ rvec, double *partials, unsigned *counter) {
    using Part = CompSum<double>::Part;
    __shared__ Part red[kBlock];
    const int t = threadIdx.x % kTB;
    const double tv = st[t].t, sg = sig[t];
    CompSum<double> acc[1];
    const int64_t m = d * kTB;
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m; e += (int64_t)gridDim.x * kBlock) {
        const int64_t j = e / kTB;
        const double q = S[e] - mu[e] * tv + sg * P[e];
        const double r = b[e] - q;
        acc[0].add(r * r);
        if (rvec && t < nv) rvec[(int64_t)t * d + j] = r;
    }
    Part mine[1];
    block_tparts<1, double>(acc, mine, red);
    if (!arrive_last_t<1>(mine, reinterpret_cast<Part *>(partials), counter, ctl)) return;
    double tot[1];
    grid_tparts<1, double>(reinterpret_cast<const Part *>(partials), gridDim.x, tot, red);
    if (threadIdx.x < kTB) {
        if (threadIdx.x < nv) out[threadIdx.x] = tot[0];
        if (threadIdx.x == 0) *counter = 0u;
    }
}

// per lane l < nv: out[2 l] = sum_i ul[i][l] v[i][l], out[2 l + 1] = the same sum of
// ul[i][l] uw[i][l] over the lane's labelled rows (y_l(i) != 0)
__global__ void __launch_bounds__(kBlock) kb_cross_dots(int64_t n, int nv, const double *__restrict__ ul,
                                                       const double *__restrict__ v, const double *__restrict__ uw,
                                                       const int8_t *__restrict__ ylab, BatchCtl *ctl, double *out,
                                                       double *partials, unsigned *counter) {
    using Part = CompSum<double>::Part;
    __shared__ Part red[kBlock * 2];
    CompSum<double> acc[2];
    const int64_t m = n * kTB;
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m; e += (int64_t)gridDim.x * kBlock) {
        acc[0].add(ul[e] * v[e]);
        if (ylab[e] != 0) acc[1].add(ul[e] * uw[e]);
    }
    Part mine[2];
    block_tparts<2, double>(acc, mine, red);
    if (!arrive_last_t<2>(mine, reinterpret_cast<Part *>(partials), counter, ctl)) return;
    double tot[2];
    grid_tparts<2, double>(reinterpret_cast<const Part *>(partials), gridDim.x, tot, red);
    if (threadIdx.x < kTB) {
        if (threadIdx.x < nv) {
            out[2 * threadIdx.x] = tot[0];
            out[2 * threadIdx.x + 1] = tot[1];
        }
        if (threadIdx.x == 0) *counter = 0u;
    }
}

// Whether op's X passes can run in fixed point (kb_fx_scan over its values; done
// once): x = x_int 2^-sx needs sx <= 24 and |x_int| < 2^bx with bx <= 10, so
// that the scaled vectors keep at least 52 bits, and sums of fewer than
// 2^(32 - bx) products (rows and columns of X shorter than that)
template <class VT>
static int fx_examine(sda_operator *op, cudaStream_t s) {
    if (op->fx_state != 0) return SDA_OK;
    int lo = 0, hi = 0, bad = 0;
    if (!std::is_same<VT, Pattern>::value && op->nnz > 0) {
        DevBuf<int> o;
        SDA_TRY(o.alloc(3));
        const int init[3] = {1 << 30, -(1 << 30), 0};
        SDA_CUDA(cudaMemcpyAsync(o.p, init, sizeof(init), cudaMemcpyHostToDevice, s));
        kb_fx_scan<VT><<<grid_elems_b(op->nnz, op->sm_count), kBlock, 0, s>>>(op->nnz, (const VT *)op->x_val_c.p, o.p);
        SDA_LAUNCHED();
        int h[3];
        SDA_CUDA(cudaMemcpyAsync(h, o.p, sizeof(h), cudaMemcpyDeviceToHost, s));
        SDA_CUDA(cudaStreamSynchronize(s));
        lo = h[0] == (1 << 30) ? 0 : h[0];
        hi = h[1] == -(1 << 30) ? 0 : h[1];
        bad = h[2];
    }
    const int sx = std::max(0, -lo), bx = hi + sx + 1;
    op->fx_sx = sx;
    op->fx_bx = bx;
    const int64_t longest = std::max(op->n, op->d);   // bounds every row and column of X
    op->fx_state = (!bad && sx <= 24 && bx <= 10 && longest < (int64_t(1) << (32 - bx))) ? 1 : -1;
    return SDA_OK;
}

// z (an FP64 block [len][kTB]) to fixed-point planes in b.fx_planes, scales in b.fx_k
static int fx_convert(sda_operator *op, BatchWs &b, int64_t len, const double *z, cudaStream_t s) {
    const int g = grid_elems_b(len * kTB, op->sm_count);
    SDA_CUDA(cudaMemsetAsync(b.fx_amax.p, 0, kTB * sizeof(unsigned long long), s));
    kb_absmax_lanes<<<g, kBlock, 0, s>>>(len, z, b.fx_amax.p);
    SDA_LAUNCHED();
    kb_to_fixed<<<g, kBlock, 0, s>>>(len, z, b.fx_amax.p, op->fx_bx, b.fx_planes.p, b.fx_k.p);
    SDA_LAUNCHED();
    return SDA_OK;
}

// U = X P - 1 c^T of an FP64 block in fixed point (one launch per plane)
template <class VT>
static int fx_rowpass(sda_operator *op, BatchWs &b, const double *p, double *ut, cudaStream_t s) {
    if (!b.grid_fx1) b.grid_fx1 = grid_for((const void *)kb_phase1_fx<BVT<VT>>, op->sm_count);
    SDA_TRY(fx_convert(op, b, b.ldw, p, s));
    for (int h = 0; h < kTB / kFxNT; ++h) {
        kb_phase1_fx<BVT<VT>><<<b.grid_fx1, kBlock, 0, s>>>(op->n, op->xr_rp.p, op->xr_col.p,
                                                           (const BVT<VT> *)op->xr_val.p,
                                                           b.fx_planes.p + h * b.ldw * kFxNT, ut, b.st.p, b.ctl.p,
                                                           h * kFxNT, op->fx_sx, b.fx_k.p);
        SDA_LAUNCHED();
    }
    return SDA_OK;
}

// S = X^T V of an FP64 block in fixed point: the head columns from shared-memory
// slices of the planes, the others with the tile pass (one launch per plane)
template <class VT>
static int fx_colpass(sda_operator *op, BatchWs &b, const double *v, double *out, cudaStream_t s) {
    SDA_TRY(fx_convert(op, b, b.n8, v, s));
    const int2 *pl = b.fx_planes.p;
    const int64_t H = op->hb.nseg;
    if (H > 0) {
        const size_t smem = (size_t)kHeadRows * kFxHNT * sizeof(int2);
        if (!b.grid_fx_head) {
            SDA_CUDA(cudaFuncSetAttribute((const void *)kb_head3a_fx<BVT<VT>>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            b.grid_fx_head = grid_for((const void *)kb_head3a_fx<BVT<VT>>, op->sm_count, smem);
        }
        const int nr = op->hb.nranges;
        const int nsplit = (int)std::max<int64_t>(
            1, std::min<int64_t>(H / 64, ((int64_t)b.head_items * b.grid_fx_head + nr - 1) / nr));
        kb_head3a_fx<BVT<VT>><<<std::min(b.grid_fx_head, nr * nsplit * (kTB / kFxHNT)), kBlock, smem, s>>>(
            op->n, b.n8, nr, (int)H, nsplit, op->hb.cp.p, op->hb.idx.p, (const BVT<VT> *)op->hb.val.p, pl,
            b.hparts.p, b.ctl.p, op->fx_sx, b.fx_k.p);
        SDA_LAUNCHED();
        const int64_t m = H * kTB;
        kb_head_reduce<double><<<(int)std::min<int64_t>((m + 31) / 32, (int64_t)op->sm_count * 8), kBlock, 0, s>>>(
            nr, m, b.hparts.p, out, b.ctl.p);
        SDA_LAUNCHED();
    }
    if (!b.grid_fx3) b.grid_fx3 = grid_for((const void *)kb_phase3a_fx<VT>, op->sm_count);
    for (int h = 0; h < kTB / kFxNT; ++h) {
        kb_phase3a_fx<VT><<<b.grid_fx3, kBlock, 0, s>>>(op->col_tail.tiles.p, op->col_tail.ntiles, op->x_cp.p + H,
                                                       op->x_row.p, (const VT *)op->x_val_c.p, pl + h * b.n8 * kFxNT,
                                                       out + H * kTB, (i128 *)b.slots.p, b.lcount.p,
                                                       op->col_tail.splits.p, b.ctl.p, h * kFxNT, op->fx_sx, b.fx_k.p);
        SDA_LAUNCHED();
    }
    return SDA_OK;
}

// the X passes of an FP64 block: fixed point where op's values allow, else FP64
template <class VT>
static int rowpass64(sda_operator *op, BatchWs &b, const double *p, double *ut, cudaStream_t s) {
    SDA_TRY(fx_examine<VT>(op, s));
    if (op->fx_state > 0) return fx_rowpass<VT>(op, b, p, ut, s);
    return rowpass_b<VT, double>(op, b, p, ut, b.grid, s);
}
template <class VT>
static int colpass64(sda_operator *op, BatchWs &b, const double *v, double *out, cudaStream_t s) {
    SDA_TRY(fx_examine<VT>(op, s));
    if (op->fx_state > 0) return fx_colpass<VT>(op, b, v, out, s);
    return colpass_b<VT, double>(op, b, v, out, b.grid, s);
}

template <class VT>
static int block64_setup(sda_operator *op, BatchWs *&B, double alpha, double omega, cudaStream_t s) {
    SDA_TRY(ensure_batch_ws<double>(op, op->bws64, 1));
    B = op->bws64;
    if (!B->grid) {
        B->grid = std::min(std::min(grid_for((const void *)kb_phase1<BVT<VT>, double>, op->sm_count),
                                    grid_for((const void *)kb_phase2<double>, op->sm_count)),
                           std::min(grid_for((const void *)kb_phase3a<VT, double>, op->sm_count),
                                    grid_for((const void *)kb_resid, op->sm_count)));
    }
    SolveState *h = B->h_st;
    memset(h, 0, sizeof(SolveState) * kTB);
    for (int v = 0; v < kTB; ++v) {
        h[v].omega = omega;
        h[v].alpha_l = alpha;
        h[v].sigma0 = 1.0;   // keeps the phase-2 step's <p, (B + sigma0) p> positive; its gamma is unused
        h[v].pp = 1.0;
    }
    SDA_CUDA(cudaMemcpyAsync(B->st.p, h, sizeof(SolveState) * kTB, cudaMemcpyHostToDevice, s));
    BatchCtl hc{};
    hc.bb = BatchBounds{op->n, op->d, B->ldw, B->n8, op->nnz, op->s_nnz, op->col.ntiles,
                        std::max(op->col.nslots, op->col_tail.nslots), std::max(op->col.nsplits, op->col_tail.nsplits),
                        (int64_t)B->part.n, (int64_t)(op->xr_col.n / 4)};
    *B->h_ctl = hc;
    SDA_CUDA(cudaMemcpyAsync(B->ctl.p, B->h_ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, s));
    return SDA_OK;
}

static int block64_check(BatchWs *B, const char *what, cudaStream_t s) {
    SDA_CUDA(cudaMemcpyAsync(B->h_ctl, B->ctl.p, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
    SDA_CUDA(cudaStreamSynchronize(s));
    if (B->h_ctl->err)
        return fail(SDA_ERR_INDEX, "%s: index check %llu failed at %llu", what,
                    (unsigned long long)(B->h_ctl->err >> 40), (unsigned long long)(B->h_ctl->err & 0xffffffffffull));
    return SDA_OK;
}

template <class VT>
static int resid_lanes_t(sda_operator *op, const ResidLane *lanes, int nl, double *r2_host, double *rvec,
                         double alpha, double omega, cudaStream_t s) {
    BatchWs *B = nullptr;
    SDA_TRY(block64_setup<VT>(op, B, alpha, omega, s));
    BView<double> bv = bview<double>(*B);
    const int64_t d = op->d, n = op->n;
    double sig[kTB] = {0};
    LaneSrc<double> wl{}, rb{}, mu{};
    LaneSrc<int8_t> yl{};
    for (int l = 0; l < nl; ++l) {
        const int t = lanes[l].t;
        sig[l] = lanes[l].sigma;
        wl.p[l] = lanes[l].w;
        rb.p[l] = lanes[l].b;
        mu.p[l] = op->mu.p + (int64_t)t * d;
        yl.p[l] = op->labels.p + (int64_t)t * n;
    }
    SDA_TRY(put_lanes(d, B->ldw, wl, bv.p, op->sm_count, s));
    SDA_TRY(put_lanes(d, B->ldw, rb, B->b.p, op->sm_count, s));
    SDA_TRY(put_lanes(d, B->ldw, mu, B->mu64.p, op->sm_count, s));
    SDA_TRY(put_lanes(n, B->n8, yl, B->ylab.p, op->sm_count, s));
    SDA_CUDA(cudaMemcpyAsync(B->sig.p, sig, sizeof(sig), cudaMemcpyHostToDevice, s));
    kb_dot_mu<<<B->grid, kBlock, 0, s>>>(d, B->mu64.p, bv.p, B->st.p, B->ctl.p, B->part.p, B->cnt.p + 0);
    SDA_LAUNCHED();
    SDA_TRY(rowpass64<VT>(op, *B, bv.p, bv.ut, s));
    kb_phase2<double><<<B->grid, kBlock, 0, s>>>(n, op->s_rp.p, op->s_col.p, op->s_val64.p, bv.ut, op->deg64.p,
                                                B->ylab.p, bv.v, B->st.p, B->ctl.p, bv.coef, 0, B->part.p,
                                                B->cnt.p + 1);
    SDA_LAUNCHED();
    SDA_TRY(colpass64<VT>(op, *B, bv.v, bv.s, s));
    kb_resid<<<B->grid, kBlock, 0, s>>>(d, nl, B->b.p, B->mu64.p, bv.s, bv.p, B->sig.p, B->st.p, B->ctl.p, B->r2.p,
                                       rvec, B->part.p, B->cnt.p + 2);
    SDA_LAUNCHED();
    SDA_CUDA(cudaMemcpyAsync(r2_host, B->r2.p, (size_t)nl * sizeof(double), cudaMemcpyDeviceToHost, s));
    return block64_check(B, "block residual", s);
}

template <class VT>
static int project_block_t(sda_operator *op, const double *Wn, int64_t nvec, double *scores, int centred, int t,
                           cudaStream_t s) {
    BatchWs *B = nullptr;
    SDA_TRY(block64_setup<VT>(op, B, 0.0, 1.0, s));
    BView<double> bv = bview<double>(*B);
    const int ge = grid_elems_b(std::max(B->ldw, B->n8) * kTB, op->sm_count);
    if (centred) {
        kb_rep<double><<<ge, kBlock, 0, s>>>(op->d, op->mu.p + (int64_t)t * op->d, B->mu64.p);
        SDA_LAUNCHED();
    }
    for (int64_t c0 = 0; c0 < nvec; c0 += kTB) {
        const int nv = (int)std::min<int64_t>(kTB, nvec - c0);
        LaneSrc<double> wl{};
        for (int v = 0; v < nv; ++v) wl.p[v] = Wn + (c0 + v) * op->d;
        SDA_TRY(put_lanes(op->d, B->ldw, wl, bv.p, op->sm_count, s));
        if (centred) {
            kb_dot_mu<<<B->grid, kBlock, 0, s>>>(op->d, B->mu64.p, bv.p, B->st.p, B->ctl.p, B->part.p, B->cnt.p + 0);
            SDA_LAUNCHED();
        }
        SDA_TRY(rowpass64<VT>(op, *B, bv.p, bv.ut, s));
        kb_unpack<<<ge, kBlock, 0, s>>>(op->n, nv, bv.ut, scores + c0 * op->n);
        SDA_LAUNCHED();
    }
    return block64_check(B, "block projection", s);
}

// The adjoint contractions of nl <= kTB targets at once (FP64, permuted order):
// per lane, out[2 l] = (X~ lam_l)^T L (X~ w_l) and out[2 l + 1] =
// (X~ lam_l)^T P_l (X~ w_l) (host), X~ = X - 1 mu_t^T of the lane's target.
template <class VT>
static int adjoint_cross_t(sda_operator *op, const int *targets, int nl, const double *W, const double *Lam,
                           double *out_host, cudaStream_t s) {
    BatchWs *B = nullptr;
    SDA_TRY(block64_setup<VT>(op, B, 1.0, 0.0, s));   // omega 0, alpha 1: phase 2 gives v = L u
    BView<double> bv = bview<double>(*B);
    const int64_t d = op->d, n = op->n;
    DevBuf<double> uw, dots;
    SDA_TRY(uw.alloc((size_t)(B->n8 * kTB)));
    SDA_TRY(dots.alloc(2 * kTB));
    {
        LaneSrc<double> mu{};
        LaneSrc<int8_t> yl{};
        for (int l = 0; l < nl; ++l) {
            mu.p[l] = op->mu.p + (int64_t)targets[l] * d;
            yl.p[l] = op->labels.p + (int64_t)targets[l] * n;
        }
        SDA_TRY(put_lanes(d, B->ldw, mu, B->mu64.p, op->sm_count, s));
        SDA_TRY(put_lanes(n, B->n8, yl, B->ylab.p, op->sm_count, s));
    }
    for (int pass = 0; pass < 2; ++pass) {
        const double *src = pass == 0 ? W : Lam;
        LaneSrc<double> wl{};
        for (int l = 0; l < nl; ++l) wl.p[l] = src + (int64_t)l * d;
        SDA_TRY(put_lanes(d, B->ldw, wl, bv.p, op->sm_count, s));
        kb_dot_mu<<<B->grid, kBlock, 0, s>>>(d, B->mu64.p, bv.p, B->st.p, B->ctl.p, B->part.p, B->cnt.p + 0);
        SDA_LAUNCHED();
        SDA_TRY(rowpass64<VT>(op, *B, bv.p, bv.ut, s));
        if (pass == 0) {
            // u_w = X~ w kept; v = L u_w
            SDA_CUDA(cudaMemcpyAsync(uw.p, bv.ut, (size_t)B->n8 * kTB * sizeof(double), cudaMemcpyDeviceToDevice, s));
            kb_phase2<double><<<B->grid, kBlock, 0, s>>>(n, op->s_rp.p, op->s_col.p, op->s_val64.p, bv.ut,
                                                        op->deg64.p, B->ylab.p, bv.v, B->st.p, B->ctl.p, bv.coef, 0,
                                                        B->part.p, B->cnt.p + 1);
            SDA_LAUNCHED();
        }
    }
    kb_cross_dots<<<B->grid, kBlock, 0, s>>>(n, nl, bv.ut, bv.v, uw.p, B->ylab.p, B->ctl.p, dots.p, B->part.p,
                                            B->cnt.p + 3);
    SDA_LAUNCHED();
    SDA_CUDA(cudaMemcpyAsync(out_host, dots.p, (size_t)nl * 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    return block64_check(B, "adjoint contractions", s);
}

// dst.p[l][j] = s[j][l] for j < len and the lanes with a destination
__global__ void __launch_bounds__(kBlock) kb_take_lanes(int64_t len, LaneSrc<double> dst, const double *__restrict__ s) {
    const int64_t m = len * kTB;
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < m; e += (int64_t)gridDim.x * kBlock) {
        const int64_t j = e / kTB;
        double *q = const_cast<double *>(dst.p[e - j * kTB]);
        if (q) q[j] = s[e];
    }
}

template <class VT>
static int xt_lanes_t(sda_operator *op, const double *const *src, int nl, double *const *dst, cudaStream_t s) {
    BatchWs *B = nullptr;
    SDA_TRY(block64_setup<VT>(op, B, 0.0, 1.0, s));
    BView<double> bv = bview<double>(*B);
    LaneSrc<double> vl{}, dl{};
    for (int l = 0; l < nl; ++l) {
        vl.p[l] = src[l];
        dl.p[l] = dst[l];
    }
    SDA_TRY(put_lanes(op->n, B->n8, vl, bv.v, op->sm_count, s));
    SDA_TRY(colpass64<VT>(op, *B, bv.v, bv.s, s));
    kb_take_lanes<<<grid_elems_b(op->d * kTB, op->sm_count), kBlock, 0, s>>>(op->d, dl, bv.s);
    SDA_LAUNCHED();
    return block64_check(B, "block X^T", s);
}

int xt_lanes(sda_operator *op, const double *const *src, int nl, double *const *dst, cudaStream_t s) {
    if (nl < 1 || nl > kTB) return fail(SDA_ERR_INVALID_ARG, "xt_lanes: %d lanes", nl);
    return with_vt_b(op->compute, [&](auto tag) -> int {
        using VT = std::remove_pointer_t<decltype(tag)>;
        return xt_lanes_t<VT>(op, src, nl, dst, s);
    });
}

int adjoint_cross(sda_operator *op, const int *targets, int nl, const double *W, const double *Lam, double *out_host,
                  cudaStream_t s) {
    if (nl < 1 || nl > kTB) return fail(SDA_ERR_INVALID_ARG, "adjoint_cross: %d lanes", nl);
    return with_vt_b(op->compute, [&](auto tag) -> int {
        using VT = std::remove_pointer_t<decltype(tag)>;
        return adjoint_cross_t<VT>(op, targets, nl, W, Lam, out_host, s);
    });
}

int resid_lanes(sda_operator *op, const ResidLane *lanes, int nl, double *r2_host, double *rvec, double alpha,
                double omega, cudaStream_t s) {
    if (nl < 1 || nl > kTB) return fail(SDA_ERR_INVALID_ARG, "resid_lanes: %d lanes", nl);
    return with_vt_b(op->compute, [&](auto tag) -> int {
        using VT = std::remove_pointer_t<decltype(tag)>;
        return resid_lanes_t<VT>(op, lanes, nl, r2_host, rvec, alpha, omega, s);
    });
}

int resid_block(sda_operator *op, int t, const double *shifts, int ns, const double *b_perm, const double *W64,
                double *out_r2, double alpha, double omega, cudaStream_t s) {
    for (int c0 = 0; c0 < ns; c0 += kTB) {
        const int nv = std::min(kTB, ns - c0);
        ResidLane rl[kTB];
        double r2[kTB];
        for (int v = 0; v < nv; ++v) rl[v] = ResidLane{t, shifts[c0 + v], b_perm, W64 + (int64_t)(c0 + v) * op->d};
        SDA_TRY(resid_lanes(op, rl, nv, r2, nullptr, alpha, omega, s));
        SDA_CUDA(cudaMemcpyAsync(out_r2 + c0, r2, (size_t)nv * sizeof(double), cudaMemcpyHostToDevice, s));
        SDA_CUDA(cudaStreamSynchronize(s));
    }
    return SDA_OK;
}

int project_block(sda_operator *op, const double *Wn, int64_t nvec, double *scores, int centred, int t,
                  cudaStream_t s) {
    return with_vt_b(op->compute, [&](auto tag) -> int {
        using VT = std::remove_pointer_t<decltype(tag)>;
        return project_block_t<VT>(op, Wn, nvec, scores, centred, t, s);
    });
}

int solve_batched(sda_operator *op, int t0, int nt, const double *const *b_perm, const double *shifts, int ns,
                  const sda_solve_opts &o, double alpha, double omega, double *w_out, sda_shift_report *rep,
                  cudaStream_t s, int *worst) {
    for (int i0 = 0; i0 < nt; i0 += kTB) {
        const int nb = std::min(kTB, nt - i0);
        double *wo = w_out ? w_out + (int64_t)i0 * ns * op->d : nullptr;
        sda_shift_report *rp = rep ? rep + (int64_t)i0 * ns : nullptr;
        int rc;
        if (op->compute == SDA_F64) {
            rc = solve_batch<double, double>(op, t0 + i0, nb, b_perm + i0, shifts, ns, o, alpha, omega, wo, rp, s,
                                             worst);
        } else {
            rc = with_vt_b(op->compute, [&](auto tag) -> int {
                using VT = std::remove_pointer_t<decltype(tag)>;
                return solve_batch<VT, float>(op, t0 + i0, nb, b_perm + i0, shifts, ns, o, alpha, omega, wo, rp, s,
                                              worst);
            });
        }
        if (rc < 0) return rc;
    }
    return SDA_OK;
}

// Single-shift solves of nl lanes (lane l: (B_{targets[l]} + betas[l] I) x_l = b[l],
// all device, permuted order) in runs of kTB lanes; the FP64 solutions go to
// x [l][D]; per-lane reports (optional).
template <class VT, class FT>
static int shift_lanes_t(sda_operator *op, const int *targets, const double *const *b, const double *betas, int nl,
                         const sda_solve_opts &o, double alpha, double omega, double *x, sda_shift_report *rep,
                         cudaStream_t s, int *worst) {
    const int64_t d = op->d;
    const bool fixed = o.fixed_iters > 0;
    const int rounds = fixed ? 0 : std::max(0, o.refine_rounds);
    const double rtol = std::isnan(o.refine_tol) || o.refine_tol <= 0.0 ? o.tol : o.refine_tol;
    const double zero = 0.0;
    for (int l0 = 0; l0 < nl; l0 += kTB) {
        const int ng = std::min(kTB, nl - l0);
        BatchLane lanes[kTB];
        for (int g = 0; g < ng; ++g) lanes[g] = BatchLane{targets[l0 + g], b[l0 + g], betas[l0 + g], o.tol};
        LaneOutcome out;
        SDA_TRY((solve_lanes<VT, FT>(op, lanes, ng, &zero, betas + l0, 1, o, alpha, omega, s, out)));
        SDA_CUDA(cudaMemcpyAsync(x + (int64_t)l0 * d, op->bws->wall.p, (size_t)ng * d * sizeof(double),
                                 cudaMemcpyDeviceToDevice, s));
        for (int g = 0; g < ng; ++g) {
            const SolveState &S = out.fin[(size_t)g];
            int st = SDA_OK;
            if (S.status != SDA_OK) st = S.status;
            else if (out.pst[(size_t)g] != SDA_OK) st = out.pst[(size_t)g];
            else if (rounds > 0) st = out.tres[(size_t)g] <= rtol ? SDA_OK : SDA_NOT_CONVERGED;
            else if (!fixed && S.sh[0].active) st = SDA_NOT_CONVERGED;
            if (st == SDA_NOT_CONVERGED && *worst == SDA_OK) *worst = SDA_NOT_CONVERGED;
            if (st < 0 && *worst >= 0) {
                *worst = st;
                fail(st, "breakdown in the solve of lane %d (target %d)", l0 + g, targets[l0 + g]);
            }
            if (rep) {
                sda_shift_report &r = rep[l0 + g];
                r.iters = S.sh[0].iters;
                r.status = st;
                r.est_residual = S.sh[0].res;
                r.true_residual = out.tres[(size_t)g];
            }
        }
    }
    SDA_CUDA(cudaStreamSynchronize(s));
    return SDA_OK;
}

int solve_shift_lanes(sda_operator *op, const int *targets, const double *const *b, const double *betas, int nl,
                      const sda_solve_opts &o, double alpha, double omega, double *x, sda_shift_report *rep,
                      cudaStream_t s, int *worst) {
    if (op->compute == SDA_F64)
        return shift_lanes_t<double, double>(op, targets, b, betas, nl, o, alpha, omega, x, rep, s, worst);
    return with_vt_b(op->compute, [&](auto tag) -> int {
        using VT = std::remove_pointer_t<decltype(tag)>;
        return shift_lanes_t<VT, float>(op, targets, b, betas, nl, o, alpha, omega, x, rep, s, worst);
    });
}

void release_batch(sda_operator *op) {
    delete op->bws;
    op->bws = nullptr;
    delete op->bws64;
    op->bws64 = nullptr;
}

}  // namespace sda
