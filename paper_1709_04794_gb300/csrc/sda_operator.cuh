// The operator object behind the opaque sda_operator handle, and the solve
// state shared between the host driver and the kernels.
#pragma once

#include "sda_common.cuh"

namespace sda {

// Per-shift recurrence state of Algorithm 3 (FP64), indexed by shift.
struct ShiftState {
    double delta;    // beta_s - sigma0 (shift relative to the base system)
    double z_prev;   // zeta_{k-1}
    double z;        // zeta_k
    double ratio;    // zeta_{k+1} / zeta_k (set when gamma_k is known)
    double g;        // gamma^s_k = gamma_k zeta_{k+1} / zeta_k
    double a;        // alpha^s_k: P_k = zeta_k r_k + alpha^s_k P_{k-1}
    double res;      // |zeta| ||r|| / ||b|| after the last update
    int32_t active;  // 0 once the shift has stopped
    int32_t iters;   // iteration count when it stopped (or so far)
};

// Scalars of the base-vector stream of one iteration, written by block 0 of
// the column pass once it has closed phase 2 (nact: shifts still active).
struct StreamParams {
    double alpha, gamma, t, sigma0;
    int32_t nact, pad;
};

// Scalars of one shifted-CG run, read by every phase kernel, written by the
// block that completes them (the last block of a phase, or block 0 of the
// column pass for phase 2's step).
struct SolveState {
    // fixed for the run
    double sigma0, omega, alpha_l, tol, bnorm, inv_bnorm;
    int32_t n_shifts, limit, fixed;
    int32_t pad0;
    const int8_t *labels;   // labels of the target being solved
    const double *mu;       // its mu_l (permuted feature order)
    const float *mu32;      // mu_l rounded to FP32
    // iteration
    int32_t k;              // iterations completed
    int32_t done;
    int32_t status;         // SDA_OK or SDA_ERR_BREAKDOWN
    int32_t nactive;
    double rr;              // <r_k, r_k>
    double alpha;           // alpha_k: p_k = r_k + alpha_k p_{k-1}
    double c;               // <mu_l, p_k>
    double pp;              // <p_k, p_k>
    double gamma;           // gamma_k = -<r_k, r_k> / <p_k, (B + sigma0) p_k>
    double gamma_prev;      // gamma_{k-1}
    double t;               // 1^T v_k
    StreamParams sp;
    ShiftState sh[kMaxShifts];
};

// A sparse matrix in column segments split into ranges of its row index, so
// that a block can keep one range's slice of the gathered vector in shared
// memory: range r holds rows [r * rb, (r + 1) * rb) with 16-bit indices local
// to it; every (range, segment) is padded with zero entries (index 0) to whole
// quads.  Warp tiles of all ranges, range after range: those of range r are
// [tile_off[r], tile_off[r + 1]).
struct RangeBlocks {
    int nranges = 0;
    int64_t rb = 0;
    int64_t nseg = 0;                 // segments (columns) per range
    int per_range = 1;                // blocks per range
    DevBuf<int64_t> cp;               // [R][nseg + 1] absolute offsets into idx / val (multiples of 4)
    DevBuf<uint16_t> idx;
    DevBuf<char> val;                 // value type of the pass; FP8 E4M3 ones for a pattern
    ColSchedule sched;
    DevBuf<int32_t> tile_off;         // [R + 1]
    int32_t slot0 = 0, lseg0 = 0;     // split chunks' slots / counters in the operator's arrays
    size_t bytes() const { return cp.bytes() + idx.bytes() + val.bytes() + sched.tiles.bytes() +
                                  sched.splits.bytes() + tile_off.bytes(); }
};

struct Workspace {
    int fp64 = -1;
    int64_t d = 0, n = 0, ldw = 0;   // ldw: D rounded up to 8 (leading dimension of D-vectors)
    int n_shifts = 0;
    int vt = -1;                     // compute dtype the grids below were sized for
    int grid1 = 0, grid2 = 0, grid3a = 0, grid3b = 0;
    int nparts = 0;                  // row ranges of the column pass (partial sums of X^T v)
    size_t colblk_smem = 0;          // its dynamic shared memory
    size_t rowhead_smem = 0;         // dynamic shared memory of the row pass (head of p_k)
    DevBuf<char> vec;        // RP[2][ldw] ({r, p} pairs), s[nparts][ldw] (pairs), ut[N8], v[N8] in the
                             // vector type (N8: N rounded up to 8)
    DevBuf<char> shift;      // W[S][ldw], P[S][ldw] in the vector type
    DevBuf<double> w64;      // the solutions in FP64 [S][D] and a residual vector [D] (permuted order)
    DevBuf<SolveState> st;
    DevBuf<double> part;     // [3][grid][4] block partials of init / phase 2 / phase 3
    DevBuf<unsigned> cnt;    // grid arrival counters of init / phase 2 / phase 3
    DevBuf<double> f64;      // FP64 scratch: b (D), w (D), q (D)
    DevBuf<double> dev_b;    // right-hand sides of the call's targets [T][D]
    DevBuf<double> adj;      // adjoint scratch: 3 D + 5 N doubles
    DevBuf<char> proj;       // scratch of the row-subset projection, grown on demand
    SolveState *h_st = nullptr;   // pinned host mirror of the state
    std::vector<cudaEvent_t> prof_ev;  // profile mode: start/end event of every phase launch of a batch
    cudaEvent_t call_ev[2] = {nullptr, nullptr};
    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0;
    cudaStream_t cap_stream = nullptr;
};

struct BatchWs;   // workspace of the batched-target solve (sda_batch.cu)

}  // namespace sda

struct sda_operator {
    int device = 0;
    int64_t n = 0, d = 0, nnz = 0, s_nnz = 0;
    int32_t n_targets = 0;
    sda_dtype compute = SDA_F64;
    double alpha = 0.0, omega = 1.0;
    bool omega_follows_alpha = true;     // built with a NaN scatter weight: omega = 1 - alpha
    bool regression = false;             // B = X^T X (sda_build_regression): no centring, alpha and omega fixed
    int sm_count = 0;

    // feature order: columns sorted by descending count (new index = rank)
    sda::DevBuf<int32_t> new_of_old, old_of_new;
    // X in CSR (columns renumbered) and CSC (new column order, rows ascending)
    sda::DevBuf<int64_t> x_rp, x_cp;
    sda::DevBuf<int32_t> x_col, x_row;
    sda::DevBuf<char> x_val_r, x_val_c;   // compute dtype (empty for PATTERN)
    // X in column-major order split into ranges of rows, for the column pass of the
    // iteration (a block keeps its range's slice of v in shared memory)
    sda::RangeBlocks xb;
    // its head columns (hb.nseg of them, possibly 0) split into ranges of kHeadRows
    // rows, for the batched column pass (hb.cp is [R][nseg + 1], no schedule)
    sda::RangeBlocks hb;
    // the other columns' tiles for the batched column pass (segments counted from hb.nseg)
    sda::ColSchedule col_tail;
    // schedule of the batched sparse passes picked by the autotuner on the first batched
    // run: resident blocks per SM of the row pass, Laplacian pass and tail column pass,
    // and work items per resident block of the head column pass (0: not tuned yet)
    int tuned[4] = {0, 0, 0, 0};
    // values of X as integers x = x_int 2^-fx_sx with |x_int| < 2^fx_bx, for the
    // exact fixed-point X passes of the FP64 block utilities; fx_state 0: not
    // examined yet, 1: they apply, -1: they do not (values too spread; FP64 passes)
    int fx_state = 0, fx_sx = 0, fx_bx = 0;
    // X in row-major order with rows padded by zero entries (column 0) to whole
    // quads, for the row pass of the iteration; features [0, xr_head) (the most
    // frequent) are gathered from shared memory there
    sda::DevBuf<int64_t> xr_rp;          // [N + 1], multiples of 4
    sda::DevBuf<int32_t> xr_col;
    sda::DevBuf<char> xr_val;            // compute dtype; FP8 E4M3 ones for PATTERN
    int xr_head = 0;
    int xr_lanes = 8;                    // lanes per row of that pass

    // graph S (CSR) and degrees D_ii; FP32 copies for the mixed path
    sda::DevBuf<int64_t> s_rp;
    sda::DevBuf<int32_t> s_col;
    sda::DevBuf<double> s_val64, deg64;
    sda::DevBuf<float> s_val32, deg32;
    // targets
    sda::DevBuf<int8_t> labels;          // [T][N]
    sda::DevBuf<double> mu;              // [T][D] mu_l, permuted order
    sda::DevBuf<float> mu32;             // [T][D] mu_l rounded to FP32 (mixed-path stream kernel)
    sda::DevBuf<double> dvec;            // [T][D] mu_+ - mu_-, permuted order
    std::vector<double> counts;          // [T][3]: l, N+, N-
    // tile schedules of the sparse passes: columns of X, rows of X, rows of S;
    // their split segments use disjoint ranges of the slots / counters below
    sda::ColSchedule col, xrow, srow;
    int32_t xrow_slot0 = 0, srow_slot0 = 0, xrow_lseg0 = 0, srow_lseg0 = 0;
    int x_lanes = 16, s_lanes = 4;        // lanes per row of the register row passes
    int grid = 0;                         // blocks of every persistent-style pass
    int64_t bytes = 0;
    // scratch of the column pass and of the FP64 reductions
    sda::DevBuf<double> slots;            // split-segment partial sums (the three schedules share them)
    sda::DevBuf<unsigned> lcount;         // split-segment arrival counters (kept at zero)
    sda::DevBuf<double> part;             // block partials of the FP64 reductions
    sda::DevBuf<unsigned> cnt;            // their arrival counters (kept at zero)
    sda::DevBuf<double> scal;             // device scalars of the FP64 operator apply

    sda::Workspace ws;
    sda::BatchWs *bws = nullptr;
    sda::BatchWs *bws64 = nullptr;   // FP64 block utilities (residual check, projection)
    sda_solve_stats stats{};
};

namespace sda {
// launchers implemented in sda_solve.cu / sda_build.cu
int op_apply_f64(const sda_operator *op, int target, double sigma, const double *p_perm, double *q_perm,
                 cudaStream_t s, double alpha, double omega);
int op_xmul_f64(const sda_operator *op, const double *w_perm, double *u, const double *csub_dev, cudaStream_t s);
int op_xtmul_f64(const sda_operator *op, const double *v, double *q, cudaStream_t s);
int permute_to_new(const sda_operator *op, const double *old_order, double *new_order, int64_t count,
                   cudaStream_t s);
int permute_to_old(const sda_operator *op, const double *new_order, double *old_order, int64_t count,
                   cudaStream_t s);
void release_workspace(sda_operator *op);
int dot_f64(const sda_operator *op, int64_t n, const double *a, const double *b, double *out, cudaStream_t s);
// ||b - (B + beta I) w||^2 of target t into *out (device), FP64, permuted order
int resid2(sda_operator *op, int t, double beta, const double *b_perm, const double *w64, double *out,
           double alpha, double omega, cudaStream_t s);
// batched targets (sda_batch.cu): targets [t0, t0 + nt) in batches sharing X and S;
// b_perm[i]: target t0 + i's right-hand side (device, permuted order)
int solve_batched(sda_operator *op, int t0, int nt, const double *const *b_perm, const double *shifts, int ns,
                  const sda_solve_opts &o, double alpha, double omega, double *w_out, sda_shift_report *rep,
                  cudaStream_t s, int *worst);
void release_batch(sda_operator *op);
// single-shift solves of nl lanes (sda_batch.cu): lane l solves (B_{targets[l]} + betas[l] I) x_l = b[l]
// (device, permuted order), runs of 16 lanes; FP64 solutions to x [nl][D]; per-lane reports (optional)
int solve_shift_lanes(sda_operator *op, const int *targets, const double *const *b, const double *betas, int nl,
                      const sda_solve_opts &o, double alpha, double omega, double *x, sda_shift_report *rep,
                      cudaStream_t s, int *worst);
// One vector of an FP64 block residual: w (device, permuted order) of target t,
// against the right-hand side b, shifted by sigma.
struct ResidLane {
    int t;
    double sigma;
    const double *b;
    const double *w;
};
// FP64 block of nl <= 16 lanes (sda_batch.cu): r2_host[l] = ||b_l - (B_{t_l} + sigma_l I) w_l||^2
// (host array, written before return); rvec (device, optional): the residual vectors [nl][D]
int resid_lanes(sda_operator *op, const ResidLane *lanes, int nl, double *r2_host, double *rvec, double alpha,
                double omega, cudaStream_t s);
// FP64 block of nl <= 16 vectors (sda_batch.cu): dst[l] = X^T src[l] (src: N-vectors, dst:
// D-vectors, device, permuted order), one column pass for all lanes
int xt_lanes(sda_operator *op, const double *const *src, int nl, double *const *dst, cudaStream_t s);
// FP64 block of nl <= 16 targets (sda_batch.cu): per lane l, out_host[2 l] = (X~ lam_l)^T L (X~ w_l),
// out_host[2 l + 1] = (X~ lam_l)^T P_l (X~ w_l), X~ = X - 1 mu_t^T (W, Lam: [nl][D] device, permuted order)
int adjoint_cross(sda_operator *op, const int *targets, int nl, const double *W, const double *Lam, double *out_host,
                  cudaStream_t s);
// FP64 blocks of 16 vectors (sda_batch.cu): out_r2[v] = ||b - (B + shifts[v] I) W64[v]||^2 of
// target t for v < ns (all device, permuted order); scores[v] = X Wn[v] (- <mu_t, Wn[v]> if centred)
int resid_block(sda_operator *op, int t, const double *shifts, int ns, const double *b_perm, const double *W64,
                double *out_r2, double alpha, double omega, cudaStream_t s);
int project_block(sda_operator *op, const double *Wn, int64_t nvec, double *scores, int centred, int t,
                  cudaStream_t s);
int64_t launch_count();
}  // namespace sda
