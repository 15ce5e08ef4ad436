/*
 * sda.h - C ABI of libsda, the GB300 (sm_103a) library for fast binary
 * semi-supervised discriminant analysis (FSDA) of Tavernier et al., arXiv
 * 1709.04794.
 *
 * The library solves, for one or many binary targets sharing one sparse
 * sample x feature matrix X (N x D, rows = samples, Sec. 2.1) and one
 * similarity graph S (N x N, Sec. 2.3-2.4), the regularised SDA systems
 *
 *     (B + beta I) w = b     for every beta of a shift sweep,
 *     B = (X - 1 mu_l^T)^T [ omega P_l + alpha L ] X                 (Alg. 7 step 4)
 *       = omega S_t^l + alpha X^T L X,   L = diag(S 1) - S,  omega = 1 - alpha  (eq. 7)
 *
 * with one shifted conjugate-gradient run per target (Algorithm 3) and the
 * centring applied implicitly as a rank-1 correction (Sec. 3.2.3), so X is
 * never densified.  mu_l is the mean labelled sample (Alg. 7 step 3), P_l
 * the diagonal 0/1 matrix of the labelled rows.  The same solver also serves
 * two operators of the paper's comparison methods: X^T X of CSR-SDA's
 * regression step (Algorithm 5; sda_build_regression) and the SDA operator
 * with X = I_N of SA-SDA (Algorithm 6; sda_build_sa).
 *
 * Conventions for every call:
 *  - Return value 0 (SDA_OK) on success, a positive warning code, or a
 *    negative error code; sda_status_string() names it and
 *    sda_last_error_detail() gives the calling thread's last message.
 *    No C++ exception crosses this boundary.
 *  - Inputs are borrowed for the duration of the call only; an operator
 *    keeps its own device copies.  Outputs are allocated by the caller.
 *  - Pointers are host or device pointers as the accompanying flag says;
 *    device pointers belong to the current CUDA device.  An operator lives
 *    on the device that was current when it was built: every call that
 *    launches work on it returns SDA_ERR_INVALID_ARG (naming both device
 *    ordinals) when another device is current, before any launch.
 *  - Device work is ordered on the caller's stream (cudaStream_t passed as
 *    void*, NULL = legacy default stream); calls that return host results
 *    synchronise that stream before returning.
 *  - An operator keeps the scratch of its calls between them, so calls on one
 *    operator must not overlap (one stream and one host thread at a time);
 *    different operators share nothing and may be used concurrently.
 */
#ifndef SDA_H
#define SDA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SDA_API __attribute__((visibility("default")))
#else
#define SDA_API
#endif

/* ---- status codes ------------------------------------------------------ */
enum {
    SDA_OK = 0,
    SDA_NOT_CONVERGED = 1,        /* warning: a shift reached max_iter before tol (see the report) */
    SDA_ERR_INVALID_ARG = -1,     /* NULL pointer, bad flag, n_shifts out of range, shift <= 0 ...  */
    SDA_ERR_SHAPE = -2,           /* inconsistent sizes between X, S, labels and vectors            */
    SDA_ERR_INDEX = -3,           /* row pointers not monotone, or a column index out of range or
                                     not strictly increasing within its row                          */
    SDA_ERR_VALUE_NOT_EXACT = -4, /* a value of X would change when stored in the compute dtype      */
    SDA_ERR_NO_POSITIVE = -5,     /* a target has no labelled positive sample: mu_+ undefined        */
    SDA_ERR_NO_NEGATIVE = -6,     /* a target has no labelled negative sample: mu_- undefined        */
    SDA_ERR_NOT_SYMMETRIC = -7,   /* S differs from S^T, or holds a negative or non-finite weight    */
    SDA_ERR_BREAKDOWN = -8,       /* <p, (B + sigma0 I) p> <= 0 or not finite during the solve       */
    SDA_ERR_TIMEOUT = -9,         /* reserved: a bounded device-side wait ran out                    */
    SDA_ERR_CUDA = -10,           /* a CUDA runtime call failed (detail in sda_last_error_detail)    */
    SDA_ERR_OOM = -11,            /* device allocation failed                                        */
    SDA_ERR_UNSUPPORTED = -12     /* a combination of options this build does not provide            */
};

/* Storage type of the values of X.  SDA_F64 selects the plain FP64 path
 * (values, vectors and sums in FP64).  The other types select the mixed
 * path: X stored in that type (binary / small-count fingerprint data is
 * exact in FP16 and FP8 e4m3), FP32 vectors and FP32 sparse sums, FP64
 * scalar recurrences, FP64 true-residual check.  SDA_PATTERN stores no
 * values at all (every stored entry is 1). */
typedef enum {
    SDA_F64 = 0,
    SDA_F32 = 1,
    SDA_F16 = 2,
    SDA_F8E4M3 = 3,
    SDA_PATTERN = 4
} sda_dtype;

/* A CSR matrix.  row_ptr has n_rows + 1 entries starting at 0 and ending at
 * nnz; col_idx has nnz entries, strictly increasing within each row and in
 * [0, n_cols).  values has nnz entries of `dtype` (SDA_F64 or SDA_F32 as
 * input types), or is NULL when dtype is SDA_PATTERN. */
typedef struct {
    int64_t n_rows, n_cols, nnz;
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const void *values;
    sda_dtype dtype;
    int32_t on_device;            /* 1: the three arrays are device pointers; 0: host pointers */
} sda_csr;

/* Labels of n_targets binary targets over the N samples, row-major
 * [n_targets][N]: +1 (positive), -1 (negative), 0 (unlabelled).  Each
 * target's labelled rows form its P_l (eq. 7). */
typedef struct {
    int32_t n_targets;
    const int8_t *labels;
    int32_t on_device;
} sda_labels;

typedef struct sda_operator sda_operator;   /* opaque, owned by the library */

/*
 * sda_build_operator - copy X and S to the device and prepare everything
 * the solves share (Alg. 7 steps 1-3): a feature order by descending column
 * count, CSR and CSC copies of X in the compute dtype, the degrees
 * D_ii = sum_j s_ij of the graph Laplacian L = D - S (Sec. 2.3), and per
 * target l, N+, N-, mu_l = X^T 1_l / l (Alg. 7 step 3) and
 * d = mu_+ - mu_- (the direction of the rank-1 right-hand side of Alg. 7
 * step 4, (X - 1 mu_l^T)^T [W 0; 0 0] X r = (N+ N- / l)(d^T r) d).
 *
 *   X              N x D sample x feature matrix (F64/F32 values, or PATTERN)
 *   S              N x N similarity graph, symmetric, weights >= 0 (diagonal ignored by L)
 *   y              labels of the targets
 *   alpha          weight of the manifold term alpha X^T L X, in [0, 1] (eq. 7)
 *   scatter_weight weight omega of the labelled total scatter; NaN selects the
 *                  paper's 1 - alpha
 *   compute        storage dtype of X on the device (see sda_dtype)
 *   cuda_stream    stream for the device work; the call synchronises it
 *   out            receives the operator; release it with sda_destroy_operator
 *
 * Errors: INVALID_ARG, SHAPE, INDEX, VALUE_NOT_EXACT, NOT_SYMMETRIC,
 * NO_POSITIVE / NO_NEGATIVE (per target), CUDA, OOM.  *out is NULL on error.
 */
SDA_API int sda_build_operator(const sda_csr *X, const sda_csr *S, const sda_labels *y,
                               double alpha, double scatter_weight, sda_dtype compute,
                               void *cuda_stream, sda_operator **out);

/*
 * sda_build_regression - the operator of the regression step of CSR-SDA
 * (Algorithm 5, line 5: shifted CG on (X^T X + beta I) w = X^T z), B = X^T X:
 * the same device layouts of X as sda_build_operator, with no graph, every
 * row weighted one and no centring.  One target (index 0).
 * sda_solve_shifts on it takes rhs_mode SDA_RHS_GIVEN (b = X^T z, computed by
 * the caller) and the operator's weights (opts alpha and scatter_weight NaN);
 * other modes return INVALID_ARG.  sda_project gives X w; sda_adjoint_grad
 * returns UNSUPPORTED.
 *
 *   X, compute, cuda_stream, out   as for sda_build_operator
 *
 * Errors: INVALID_ARG, SHAPE, INDEX, VALUE_NOT_EXACT, CUDA, OOM.  *out is
 * NULL on error.
 */
SDA_API int sda_build_regression(const sda_csr *X, sda_dtype compute_values, void *cuda_stream,
                                 sda_operator **out);

/*
 * sda_build_sa - the operator of SA-SDA (Algorithm 6): the SDA operator with
 * the identity I_N as the data matrix, B = (I - 1 1_l^T / l)^T M, M = omega P_l
 * + alpha L, over N-vectors (= M - omega 1_l 1_l^T / l, symmetric, since
 * M 1 = omega 1_l).  The canonical right-hand side d = 1_+ / N+ - 1_- / N- is
 * the direction of Algorithm 6's [W 0; 0 0] r for any r orthogonal to 1_l; the
 * solution z is the rating itself (s = z).  Every solve option applies.
 *
 *   S, y, alpha, scatter_weight, compute, cuda_stream, out
 *                  as for sda_build_operator (X is I_N, built internally)
 *
 * Errors: as for sda_build_operator.
 */
SDA_API int sda_build_sa(const sda_csr *S, const sda_labels *y, double alpha, double scatter_weight,
                         sda_dtype compute_values, void *cuda_stream, sda_operator **out);

/* Right-hand side of the solve (Alg. 7 step 4). */
enum {
    SDA_RHS_CANONICAL = 0,  /* b = d = mu_+ - mu_- (positives score high)                          */
    SDA_RHS_FROM_R = 1,     /* b = (X - 1 mu_l^T)^T [W 0; 0 0] X r for the given r in R^D
                               (= (N+ N- / l)(d^T r) d); `rhs` holds r (D doubles, shared by all
                               targets of the call)                                                */
    SDA_RHS_GIVEN = 2       /* b given in `rhs`: [target_count][D] doubles                          */
};

typedef struct {
    double tol;             /* shift s stops when |zeta_s| ||r|| < tol ||b|| (Alg. 3, relative)     */
    int32_t max_iter;       /* iteration cap for every shift                                       */
    int32_t fixed_iters;    /* > 0: run exactly this many iterations, ignore tol (Sec. 5.2: 70);   */
                            /* a target whose residual vanishes exactly stops there (SDA_OK)       */
    int32_t rhs_mode;       /* SDA_RHS_*                                                           */
    const double *rhs;      /* see rhs_mode; NULL for SDA_RHS_CANONICAL                            */
    int32_t rhs_on_device;  /* 1: `rhs` is a device pointer                                        */
    int32_t target_begin;   /* first target solved by this call                                    */
    int32_t target_count;   /* number of targets solved by this call (-1: all from target_begin)   */
    int32_t check_residual; /* 1: compute the FP64 true relative residual of every shift (its X    */
                            /* passes exact in integers where X's values allow, see info)          */
    int32_t out_on_device;  /* 1: w_out is a device pointer; 0: host pointer                       */
    int32_t use_graph;      /* 1: replay the iteration loop as captured CUDA graphs                */
    int32_t iter_batch;     /* iterations launched between two host convergence checks (0: auto)   */
    int32_t profile;        /* 1: launch without graphs and time every phase kernel with CUDA
                               events (sda_get_solve_stats); slower, for measurement only         */
    double alpha;           /* NaN: the operator's alpha; else this call's alpha in [0, 1] (eq. 7)  */
    double scatter_weight;  /* NaN: 1 - alpha if the operator was built with a NaN scatter weight,
                               else the operator's omega; else this call's omega >= 0              */
    int32_t refine_rounds;  /* > 0: per-shift refinement (no paper counterpart): while a shift's FP64
                               true residual exceeds refine_tol, solve (B + beta I) c = b - (B + beta I) w
                               in the iteration's precision and add c in FP64, at most this many times;
                               a shift still above refine_tol reports SDA_NOT_CONVERGED             */
    int32_t batch_targets;  /* 1: solve the call's targets in batches of 16 that share every pass over
                               X and S (vectors stored target-contiguous; no paper counterpart);
                               0: one target after another.  With refine_rounds > 0 the correction
                               solves of up to 16 (target, shift) pairs of a batch share one run too */
    double refine_tol;      /* target FP64 true relative residual (NaN or <= 0: tol)                */
    int32_t shift_form;     /* how the batched path forms every shift's solution: SDA_SHIFTS_*    */
} sda_solve_opts;

/* Shift forms of the batched path (opts.batch_targets = 1).  The single-target
 * path always runs the recurrences (SDA_SHIFTS_BASIS there: SDA_ERR_UNSUPPORTED). */
enum {
    SDA_SHIFTS_AUTO = 0,        /* the stored basis when every shift is solved at once (n_shifts > 1) and
                                   (limit + 1) x D x 16 basis values fit in 40 % of the free device
                                   memory, else the recurrences                                         */
    SDA_SHIFTS_RECURRENCE = 1,  /* Algorithm 3: every active shift's W and P updated every iteration  */
    SDA_SHIFTS_BASIS = 2        /* Lanczos form (Sec. 3.2.1, eqs. for T and the shifted solve): the base
                                   residuals r_0 .. r_{K-1} are kept (the basis V up to scaling), the
                                   tridiagonal T_K of the base system comes from the CG scalars, each shift
                                   solves (T_{K_s} + (beta_s - sigma0) I) y = ||b|| e_1 in FP64 and
                                   W_s = V y is formed once after the run (K_s: the shift's stop)        */
};

/* Fills *opt with: tol 1e-6, max_iter 10000, fixed_iters 0, canonical RHS,
 * all targets, FP64 residual check on, device output, graphs on, auto batch,
 * the operator's alpha and omega, no refinement, SDA_SHIFTS_AUTO. */
SDA_API void sda_default_opts(sda_solve_opts *opt);

/* Per target and shift outcome of sda_solve_shifts. */
typedef struct {
    int32_t iters;          /* iteration at which the shift stopped (Alg. 3 stop test)             */
    int32_t status;         /* SDA_OK, SDA_NOT_CONVERGED or SDA_ERR_BREAKDOWN                      */
    double est_residual;    /* |zeta| ||r|| / ||b|| when it stopped                                */
    double true_residual;   /* ||b - (B + beta I) w|| / ||b|| in FP64, or -1 when not computed     */
} sda_shift_report;

/*
 * sda_solve_shifts - solve (B + beta_s I) w_s = b for every shift of every
 * target in the call's range with one shifted-CG run per target
 * (Algorithm 3; base system B + sigma0 I, sigma0 = min beta, recurrences on
 * the relative shifts; the shift coefficient uses the new CG coefficient,
 * alpha^b_{i+1} = alpha_{i+1} (zeta^b_{i+1} / zeta^b_i)^2).
 *
 *   shifts     n_shifts values > 0 (host), 1 <= n_shifts <= 64
 *   opt        options (NULL: sda_default_opts)
 *   w_out      [target_count][n_shifts][D] doubles in the caller's feature order, or NULL
 *   report     host array [target_count][n_shifts], or NULL
 *
 * D is the operator's number of features (N for an operator from
 * sda_build_sa).  An operator from sda_build_regression takes rhs_mode
 * SDA_RHS_GIVEN and opts alpha / scatter_weight NaN, else INVALID_ARG.
 *
 * Returns SDA_OK, SDA_NOT_CONVERGED (some shift hit max_iter; its report
 * says which), or an error: INVALID_ARG, SHAPE, BREAKDOWN, CUDA, OOM.
 * Synchronises the stream.
 */
SDA_API int sda_solve_shifts(sda_operator *op, const double *shifts, int32_t n_shifts,
                             const sda_solve_opts *opt, double *w_out, sda_shift_report *report,
                             void *cuda_stream);

/*
 * sda_adjoint_grad - gradient of a loss of held-out scores with respect to
 * (alpha, beta) by one adjoint solve on the same symmetric operator (not in
 * the paper; a training-style use of the solve).
 *
 * w solves (B(alpha) + beta I) w = b (Algorithm 3); the held-out scores are
 * s_h = (X_h - 1 mu_l^T) w for the rows `rows`; the caller passes
 * g = d loss / d s_h.  With lambda solving (B + beta I) lambda = (X_h - 1 mu_l^T)^T g,
 *   d loss / d beta  = -lambda^T w
 *   d loss / d alpha = -lambda^T (dB/dalpha) w
 *                    = -[(X~ lambda)^T L (X~ w) - c (X~ lambda)^T P_l (X~ w)],
 * X~ = X - 1 mu_l^T, c = 1 when omega follows 1 - alpha, else 0 (eq. 7).
 *
 *   target, alpha, beta  the point of w (alpha NaN: the operator's)
 *   w                    D doubles, device, caller's feature order
 *   dloss_ds, rows       n_rows doubles and n_rows int64 row ids (device); repeated
 *                        rows add up
 *   opt                  tolerance and iteration cap of the adjoint solve (NULL:
 *                        defaults with tol 1e-10); its alpha/scatter_weight are ignored
 *   d_alpha, d_beta      host doubles receiving the gradient
 *   lambda_out           D doubles (device, caller order) receiving lambda, or NULL
 * Errors: INVALID_ARG (a row out of range), BREAKDOWN, CUDA, OOM; SDA_NOT_CONVERGED
 * when the adjoint solve hit its cap.  Synchronises the stream.
 */
SDA_API int sda_adjoint_grad(sda_operator *op, int32_t target, double alpha, double beta, const double *w,
                             const double *dloss_ds, const int64_t *rows, int64_t n_rows,
                             const sda_solve_opts *opt, double *d_alpha, double *d_beta, double *lambda_out,
                             void *cuda_stream);

/*
 * sda_adjoint_grad_batched - sda_adjoint_grad for many targets at once (not
 * in the paper): target targets[i] at (alpha, betas[i]) with the solution
 * W[i] and the held-out rows rows[row_off[i] .. row_off[i + 1]) with their
 * loss gradients dloss_ds[same range].  The adjoint solves
 * (B_t + beta_i I) lambda_i = (X_h - 1 mu_l^T)^T g_i of up to 16 targets share
 * one batched run (the batched path of sda_solve_shifts, one shift per lane);
 * the contractions are FP64 per target, as in sda_adjoint_grad.
 *
 *   n_targets            number of gradients (0: nothing to do)
 *   targets, betas       host arrays [n_targets] (targets may repeat)
 *   alpha                the common alpha (NaN: the operator's)
 *   W                    [n_targets][D] doubles, device, caller's feature order
 *   dloss_ds, rows       device arrays of row_off[n_targets] doubles / int64 row ids
 *   row_off              host int64 [n_targets + 1], row_off[0] = 0, non-decreasing
 *   opt                  tolerance, cap, fixed_iters, refinement of the adjoint solves
 *                        (NULL: defaults with tol 1e-10); its alpha/scatter_weight,
 *                        rhs and target range are ignored
 *   d_alpha, d_beta      host [n_targets]
 *   lambda_out           [n_targets][D] doubles (device, caller order), or NULL
 *   report               host [n_targets] reports of the adjoint solves, or NULL
 * Errors: INVALID_ARG (a row or target out of range, bad offsets), UNSUPPORTED
 * (regression operator), BREAKDOWN, CUDA, OOM; SDA_NOT_CONVERGED when an
 * adjoint solve hit its cap.  Synchronises the stream.
 */
SDA_API int sda_adjoint_grad_batched(sda_operator *op, int32_t n_targets, const int32_t *targets, double alpha,
                                     const double *betas, const double *W, const double *dloss_ds,
                                     const int64_t *rows, const int64_t *row_off, const sda_solve_opts *opt,
                                     double *d_alpha, double *d_beta, double *lambda_out,
                                     sda_shift_report *report, void *cuda_stream);

/*
 * sda_heldout_logistic - choose the shift of each target on its held-out rows.
 * The paper picks the regularisation beta on held-out folds (Sec. 5); the
 * criterion here is the logistic loss of the ratings, the loss whose
 * gradient sda_adjoint_grad(_batched) takes:
 *     loss[t][s] = (1/m_t) sum_h log(1 + exp(-y_h s_{t,s,h}))   (m_t rows of target t)
 *     best[t]    = the s of least loss[t][s] (the smallest such s on ties; NaN
 *                  losses are never least unless all are NaN, then 0)
 *     g_h        = d loss[t][best[t]] / d s_h = -y_h / (1 + exp(y_h s_{t,best,h})) / m_t
 * FP64; every sum is taken in a fixed order, so repeated calls give the same bits.
 *
 *   n_targets, n_shifts  >= 0 and >= 1
 *   row_off              host int64 [n_targets + 1], row_off[0] = 0, non-decreasing:
 *                        target t owns held-out rows [row_off[t], row_off[t + 1])
 *   scores               device doubles [n_shifts * row_off[n_targets]]; target t's ratings
 *                        start at n_shifts * row_off[t], laid out [n_shifts][m_t] (the
 *                        layout sda_project_rows writes for one target)
 *   y                    device doubles [row_off[n_targets]]: the rows' labels (+1 / -1)
 *   loss                 device doubles [n_targets][n_shifts]
 *   best                 device int32 [n_targets]
 *   g                    device doubles [row_off[n_targets]]
 * A target with no rows gets loss 0 for every shift and best 0.  Errors:
 * INVALID_ARG (bad sizes or offsets, a NULL array), CUDA.  Does not
 * synchronise the stream.
 */
SDA_API int sda_heldout_logistic(int32_t n_targets, int32_t n_shifts, const int64_t *row_off, const double *scores,
                                 const double *y, double *loss, int32_t *best, double *g, void *cuda_stream);

/*
 * sda_knn_graph - the similarity graph S of Sec. 2.4 built on the device from
 * the samples: s_ij = Tanimoto (Jaccard) similarity of the binary supports of
 * rows i and j of X, |x_i and x_j| / |x_i or x_j| (Tanimoto on fingerprints,
 * Sec. 5.1); the edges are the union of every row's k nearest rows (the
 * undirected kNN graph of Sec. 2.4), ranked by (similarity descending, row
 * index ascending); similarity 0 never makes an edge, and with threshold > 0
 * neither does a similarity below it (the similarity threshold of Sec. 2.4;
 * Sec. 5.2 uses Tanimoto >= 0.4).  Candidates of row i are the rows sharing a
 * feature whose column count is <= cap (cap >= N: every shared feature, the
 * exact kNN graph).  The result is symmetric with a zero diagonal and is a
 * valid S for sda_build_operator.
 *
 *   X          N x D (values ignored: the binary support counts); host or device arrays
 *   k          neighbours per row, 1 .. 32
 *   cap        column-count limit of the features that propose candidates (>= 1)
 *   threshold  smallest similarity kept, in [0, 1]
 *   row_ptr    device int64 [N + 1]; col_out, val_out: device int32 / double [capacity]
 *   nnz_out    host: the entries of S (also when they exceed capacity)
 * Rows are sorted by column.  Errors: INVALID_ARG, SHAPE (sizes, or an output
 * smaller than the graph: *nnz_out says how large), INDEX, UNSUPPORTED (a row
 * of more than 1,024 features), CUDA, OOM.  Synchronises the stream.
 */
SDA_API int sda_knn_graph(const sda_csr *X, int32_t k, int64_t cap, double threshold, int64_t *row_ptr,
                          int32_t *col_out, double *val_out, int64_t capacity, int64_t *nnz_out, void *cuda_stream);

/*
 * sda_project - ratings s = X w of the samples (Sec. 4, Alg. 7 step 5), or
 * the centred ratings (X - 1 mu_l^T) w when `centred` is 1 (uses mu_l of
 * `target`).  FP64 sums.
 *
 *   w        [n_vec][D] doubles in the caller's feature order (device)
 *   scores   [n_vec][N] doubles (device)
 */
SDA_API int sda_project(const sda_operator *op, const double *w, int64_t n_vec, double *scores,
                        int32_t centred, int32_t target, void *cuda_stream);

/*
 * sda_project_rows - the ratings of a subset of the samples only (Sec. 4,
 * Alg. 7 step 5 restricted to the rows one scores, e.g. held-out compounds):
 * scores[v][h] = (X w_v)_{rows[h]}, or the centred (X w_v)_{rows[h]} - mu_l^T w_v
 * when `centred` is 1 (mu_l of `target`).  FP64 sums.
 *
 *   w        [n_vec][D] doubles in the caller's feature order (device)
 *   rows     n_rows row ids (device int64); repeated ids are allowed
 *   scores   [n_vec][n_rows] doubles (device)
 * The operator keeps the call's scratch (n_vec D doubles and a little more)
 * for later calls.  Errors: INVALID_ARG (a row id outside [0, N), bad
 * argument), CUDA, OOM.  Synchronises the stream.
 */
SDA_API int sda_project_rows(const sda_operator *op, const double *w, int32_t n_vec, const int64_t *rows,
                             int64_t n_rows, double *scores, int32_t centred, int32_t target, void *cuda_stream);

/*
 * sda_operator_apply - q = (B + sigma I) p for one target in FP64 (the
 * operator of Alg. 7 step 4 in its centred symmetric form
 * (X - 1 mu_l^T)^T M (X - 1 mu_l^T), equal to the paper's form because
 * M 1 = omega 1_l and (X - 1 mu_l^T)^T 1_l = 0).  p and q are device arrays
 * of D doubles in the caller's feature order.
 */
SDA_API int sda_operator_apply(const sda_operator *op, int32_t target, double sigma,
                               const double *p, double *q, void *cuda_stream);

/*
 * sda_operator_apply_static - the same q = (B + sigma I) p as
 * sda_operator_apply, for callers that cannot allocate device memory: a
 * host application whose device memory is entirely owned by its own pool
 * allocator (a cudaMalloc from the library would compete with it for the
 * same memory), and latency-critical loops where the implicit device
 * synchronisation of cudaMalloc / cudaFree is not acceptable.  The paper has
 * no counterpart; this is an interface convenience.
 *
 * Every per-call buffer lives in one file-scope device array of
 * SDA_STATIC_SCRATCH_DOUBLES doubles (8 MiB) that every GPU loading the
 * library holds until the process exits; the call allocates nothing and
 * does not synchronise the stream.  The operator must satisfy
 *     2 D + 2 N + (reduction and split-segment slots) <= SDA_STATIC_SCRATCH_DOUBLES,
 * otherwise the call returns SDA_ERR_SHAPE and names the size it needed.
 * All calls share the array and it keeps the last call's contents (the call
 * clears the counters that must start at zero itself), so calls that overlap
 * on the GPU (different streams, or different host threads) race and must be
 * serialised by the caller.  The first call on a device looks the array's
 * address up with that device current (which loads the library's device code
 * on that device).  p and q
 * are device arrays of D doubles in the caller's feature order; errors as
 * sda_operator_apply.
 */
#define SDA_STATIC_SCRATCH_DOUBLES (1 << 20)

SDA_API int sda_operator_apply_static(const sda_operator *op, int32_t target, double sigma,
                                      const double *p, double *q, void *cuda_stream);

/* Counters of the last sda_solve_shifts call on an operator. */
typedef struct {
    int64_t iterations;        /* Krylov iterations summed over the call's targets (batched mode:
                                  over its batches, each counting its slowest target)               */
    int64_t shift_iterations;  /* sum over targets and shifts of the iterations each shift ran      */
    int64_t launches[5];       /* kernel launches: [0] start, [1] X rows (X p), [2] S rows (L u),
                                  [3] X columns (X^T v), [4] vector and shift-state update          */
    double ms[5];              /* device time of those launches in ms (profile mode, else 0)        */
    double solve_ms;           /* device time of the whole call in ms                               */
    int32_t shift_form;        /* SDA_SHIFTS_RECURRENCE or SDA_SHIFTS_BASIS: the form the call's first
                                  batched run used (RECURRENCE on the single-target path)              */
    int32_t basis_slots;       /* stored-basis form: basis vectors (iterations) kept by that run         */
} sda_solve_stats;

SDA_API int sda_get_solve_stats(const sda_operator *op, sda_solve_stats *stats);

/* Number of kernels libsda has launched in this process (graph replays count
 * every kernel of the graph).  Instrumentation for benchmarks. */
SDA_API int64_t sda_kernel_launch_count(void);

/* Sizes of an operator. */
typedef struct {
    int64_t n_rows, n_cols, nnz, graph_nnz;
    int32_t n_targets;
    sda_dtype compute;
    double alpha, omega;
    int64_t device_bytes;   /* device memory held by the operator (without solve workspace) */
    /* layouts of the iteration's sparse passes: */
    int32_t col_ranges;     /* ranges of rows of the column pass (X^T v partial sums per feature) */
    int32_t row_head;       /* leading features the row pass gathers from shared memory */
    int64_t col_entries;    /* entries of the column-pass layout, padding to quads included */
    int64_t row_entries;    /* entries of the row-pass layout, padding to quads included */
    /* head of the batched column pass (the most frequent columns in ranges of rows): */
    int32_t head_cols;      /* head columns (0: none; every column takes the tile pass) */
    int32_t head_ranges;    /* ranges of rows */
    int64_t head_entries;   /* entries of its layout, padding to quads included */
    /* schedule of the batched sparse passes picked by the autotuner on the operator's
       first batched run (0 until then): resident blocks per SM of the row pass, the
       Laplacian pass and the tail column pass, and work items per resident block of
       the head column pass (-1: no head pass, every column through the tile pass) */
    int32_t tuned[4];
    /* X passes of the FP64 residual checks, projections and block utilities: 1 when
       they run in exact fixed point (every value of X is x_int 2^-x_frac_bits with
       |x_int| < 2^x_int_bits, x_frac_bits <= 24, x_int_bits <= 10, and N, D <
       2^(32 - x_int_bits): integer products and sums, exact, one rounding to FP64
       per result), -1 when they run in FP64 arithmetic, 0 until the operator's
       first such pass */
    int32_t exact_x_passes;
    int16_t x_frac_bits, x_int_bits;
} sda_operator_info;

SDA_API int sda_get_operator_info(const sda_operator *op, sda_operator_info *info);

/* Per-target counts (l, N+, N-) as doubles, host array [n_targets][3]. */
SDA_API int sda_get_target_counts(const sda_operator *op, double *counts);

/* Releases the operator and its device memory (NULL is a no-op). */
SDA_API void sda_destroy_operator(sda_operator *op);

/* Static string naming a status code. */
SDA_API const char *sda_status_string(int code);

/* Copies the calling thread's last error message into buf (NUL-terminated,
 * truncated to len); returns the code of that error (0 if none). */
SDA_API int sda_last_error_detail(char *buf, int len);

#ifdef __cplusplus
}
#endif

#endif /* SDA_H */
