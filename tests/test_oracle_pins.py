"""Pins of the FP64 CPU oracle to facts fixed by the paper and by mathematics.

Each test names the passage it follows.  None of them re-types the oracle's
own formula: the dense checks build B from the sample sums of eq. (7) and
the regulariser of Sec. 2.3, the eigenproblem goes through a library
generalised-eigen routine, and the rest are closed forms, invariances,
special cases and brute force.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_1709_04794_gb300 import synth


def _dense(prob, t=0):
    return oracle.dense_x(prob.x_ptr, prob.x_col, prob.x_val, prob.d)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# --------------------------------------------------------------------------
# Operator (eq. 7, Alg. 7 step 4, Sec. 3.2.3)
# --------------------------------------------------------------------------

def test_operator_equals_sample_sum_definition(tiny):
    """B p from the matrix-free paper form equals (1-a) S_t^l + a X^T L X built from
    sums over samples (eq. 7) and over graph edges (regulariser, Sec. 2.3)."""
    o = oracle.from_problem(tiny)
    X = _dense(tiny)
    B = oracle.dense_operator(X, tiny.s_ptr, tiny.s_col, tiny.s_val, tiny.labels[0], tiny.alpha)
    rng = np.random.default_rng(0)
    for sigma in (0.0, 0.37):
        p = rng.standard_normal(tiny.d)
        assert _rel(o.apply(p, sigma), B @ p + sigma * p) < 1e-12


def test_operator_symmetric_psd(cfg1):
    """B is symmetric positive semi-definite (Sec. 3.2.1: 'symmetric ... SDA')."""
    o = oracle.from_problem(cfg1)
    rng = np.random.default_rng(1)
    for _ in range(3):
        x, y = rng.standard_normal(cfg1.d), rng.standard_normal(cfg1.d)
        bx, by = o.apply(x), o.apply(y)
        assert abs(x @ by - bx @ y) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(by)
        assert x @ bx >= -1e-12 * (x @ x)


def test_centred_operator_kills_nondiscriminative_direction(tiny):
    """Sec. 3.2.3: with centring around mu_l, the vector w_nd with X w_nd = 1 is in
    the null space: B w_nd = 0.  Make w_nd exist by adding an all-ones feature."""
    n, d = tiny.n, tiny.d
    counts = np.diff(tiny.x_ptr)
    x_ptr = np.concatenate([[0], np.cumsum(counts + 1)]).astype(np.int64)
    x_col = np.empty(x_ptr[-1], dtype=np.int32)
    x_val = np.empty(x_ptr[-1])
    for i in range(n):
        a, b = tiny.x_ptr[i], tiny.x_ptr[i + 1]
        x_col[x_ptr[i]:x_ptr[i + 1]] = np.concatenate([tiny.x_col[a:b], [d]])
        x_val[x_ptr[i]:x_ptr[i + 1]] = np.concatenate([tiny.x_val[a:b], [1.0]])
    o = oracle.Oracle(x_ptr, x_col, x_val, tiny.s_ptr, tiny.s_col, tiny.s_val, tiny.labels[0],
                      d + 1, tiny.alpha)
    e = np.zeros(d + 1)
    e[d] = 1.0
    q = o.apply(e)
    scale = np.linalg.norm(o.apply(np.random.default_rng(2).standard_normal(d + 1)))
    assert np.linalg.norm(q) <= 1e-13 * scale
    # without the centring correction it is not in the null space: the uncentred
    # operator X^T M X maps w_nd to (1 - alpha) X^T 1_l = (1 - alpha) l mu_l != 0
    X = oracle.dense_x(x_ptr, x_col, x_val, d + 1)
    y = tiny.labels[0]
    unc = (1 - tiny.alpha) * X.T @ ((y != 0) * (X @ e))
    assert np.linalg.norm(unc) > 1.0


def test_paper_form_equals_symmetric_centred_form(tiny):
    """(X - 1 mu^T)^T M X = (X - 1 mu^T)^T M (X - 1 mu^T) because M 1 = (1-a) 1_l
    (L 1 = 0, Sec. 2.5.2) and (X - 1 mu^T)^T 1_l = 0."""
    o = oracle.from_problem(tiny)
    X = _dense(tiny)
    y = tiny.labels[0]
    mu = X[y != 0].mean(axis=0)
    Xc = X - mu
    n = tiny.n
    S = np.zeros((n, n))
    S[np.repeat(np.arange(n), np.diff(tiny.s_ptr)), tiny.s_col] = tiny.s_val
    L = np.diag(S.sum(axis=1)) - S
    M = (1 - tiny.alpha) * np.diag((y != 0).astype(float)) + tiny.alpha * L
    p = np.random.default_rng(3).standard_normal(tiny.d)
    assert _rel(o.apply(p), Xc.T @ (M @ (Xc @ p))) < 1e-12


def test_class_means(tiny):
    """l mu_l = X^T 1_l (Alg. 7 step 3) and the class means, against dense sums."""
    o = oracle.from_problem(tiny)
    X = _dense(tiny)
    y = tiny.labels[0]
    mu, mp, mn, cnt = o.class_means()
    assert np.allclose(mu, X[y != 0].mean(axis=0), rtol=0, atol=1e-14)
    assert np.allclose(mp, X[y > 0].mean(axis=0), rtol=0, atol=1e-14)
    assert np.allclose(mn, X[y < 0].mean(axis=0), rtol=0, atol=1e-14)
    assert list(cnt) == [(y != 0).sum(), (y > 0).sum(), (y < 0).sum()]


def test_rhs_rank_one_closed_form(tiny):
    """Alg. 7 step 4 RHS (X - 1 mu^T)^T [W 0; 0 0] X r equals (N+ N- / l)(d^T r) d:
    the between-class scatter of two classes has rank one (Sec. 2.2.1, Sec. 3.1)."""
    o = oracle.from_problem(tiny)
    _, mp, mn, cnt = o.class_means()
    dvec = mp - mn
    r = synth.random_r(5, tiny.d)
    b = o.rhs_from_r(r)
    expect = cnt[1] * cnt[2] / cnt[0] * (dvec @ r) * dvec
    assert _rel(b, expect) < 1e-12


# --------------------------------------------------------------------------
# Solvers (Alg. 2, Alg. 3, eq. 10-12)
# --------------------------------------------------------------------------

def test_shifted_cg_equals_dense_direct_solve(tiny):
    """w_beta = (B + beta I)^{-1} b by Cholesky of the dense B, for every shift."""
    o = oracle.from_problem(tiny)
    X = _dense(tiny)
    B = oracle.dense_operator(X, tiny.s_ptr, tiny.s_col, tiny.s_val, tiny.labels[0], tiny.alpha)
    b = o.rhs_canonical()
    res = o.shifted_cg(b, tiny.shifts, tol=1e-14, max_iter=5000)
    assert res.status == 0
    for s, beta in enumerate(tiny.shifts):
        A = B + beta * np.eye(tiny.d)
        w = scipy.linalg.cho_solve(scipy.linalg.cho_factor(A), b)
        kappa = np.linalg.cond(A)
        assert _rel(res.W[s], w) < max(1e-12, 1e-14 * kappa * 10), (beta, kappa)


def test_cg_equals_dense_direct_solve(tiny):
    o = oracle.from_problem(tiny)
    X = _dense(tiny)
    B = oracle.dense_operator(X, tiny.s_ptr, tiny.s_col, tiny.s_val, tiny.labels[0], tiny.alpha)
    b = o.rhs_canonical()
    beta = tiny.shifts[1]
    w, it, r, rc = o.cg(b, beta, tol=1e-14, max_iter=5000)
    assert rc == 0
    assert _rel(w, np.linalg.solve(B + beta * np.eye(tiny.d), b)) < 1e-10


def test_generalised_eigenproblem_rank_one(tiny):
    """Eq. (7)/(10): S_B v = lambda (B + beta I) v with rank-1 S_B has one nonzero
    eigenvalue (N+N-/l) d^T (B+beta I)^{-1} d, eigenvector ∝ the solve's w."""
    o = oracle.from_problem(tiny)
    X = _dense(tiny)
    y = tiny.labels[0]
    B = oracle.dense_operator(X, tiny.s_ptr, tiny.s_col, tiny.s_val, y, tiny.alpha)
    SB = oracle.dense_between(X, y)
    beta = tiny.shifts[2]
    lam, V = scipy.linalg.eigh(SB, B + beta * np.eye(tiny.d))
    b = o.rhs_canonical()
    res = o.shifted_cg(b, [beta], tol=1e-14, max_iter=5000)
    w = res.W[0]
    _, _, _, cnt = o.class_means()
    lam_max = cnt[1] * cnt[2] / cnt[0] * (b @ w)
    assert abs(lam[-1] - lam_max) <= 1e-10 * lam_max
    assert np.all(np.abs(lam[:-1]) <= 1e-10 * lam_max)
    v = V[:, -1]
    cos = abs(v @ w) / (np.linalg.norm(v) * np.linalg.norm(w))
    assert cos > 1 - 1e-12


def test_subspace_iteration_converges_in_one_step(tiny):
    """Sec. 3.1 / Alg. 1: with j = C - 1 = 1 one step of subspace iteration gives the
    eigenvector: V solves (B + beta I) V = S_B R for a random R."""
    o = oracle.from_problem(tiny)
    X = _dense(tiny)
    y = tiny.labels[0]
    B = oracle.dense_operator(X, tiny.s_ptr, tiny.s_col, tiny.s_val, y, tiny.alpha)
    SB = oracle.dense_between(X, y)
    beta = tiny.shifts[0]
    R = synth.random_r(9, tiny.d)
    V = np.linalg.solve(B + beta * np.eye(tiny.d), SB @ R)
    w = o.shifted_cg(o.rhs_canonical(), [beta], tol=1e-14, max_iter=5000).W[0]
    cos = abs(V @ w) / (np.linalg.norm(V) * np.linalg.norm(w))
    assert cos > 1 - 1e-12


@pytest.mark.parametrize("k", [1, 2, 3, 5, 12, 40])
def test_shifted_iterates_equal_per_shift_cg(cfg1, k):
    """Sec. 3.2.2: the Krylov space does not depend on the shift, so after k steps the
    shifted-CG iterate of every shift equals k steps of plain CG (Alg. 2) on B + beta I.
    Fails with the printed alpha_i in the shift-coefficient update (index slip)."""
    o = oracle.from_problem(cfg1)
    b = o.rhs_canonical()
    res = o.shifted_cg(b, cfg1.shifts, fixed_iters=k)
    assert res.status == 0
    for s, beta in enumerate(cfg1.shifts):
        w, it, _, rc = o.cg(b, beta, fixed_iters=k)
        assert rc == 0 and it == k
        # exact in exact arithmetic; FP64 rounding grows with k on the ill-conditioned shifts
        tol = 1e-10 if k <= 12 else 1e-7
        assert _rel(res.W[s], w) < tol, (k, beta, _rel(res.W[s], w))


def test_residual_collinear_and_monotone_in_shift(cfg1):
    """r^beta_k = zeta^beta_k r_k: the explicit residual of every shift has norm
    |zeta| ||r|| (Alg. 3 stop test), and |zeta| does not grow with the shift."""
    o = oracle.from_problem(cfg1)
    b = o.rhs_canonical()
    for k in (4, 15, 30):
        res = o.shifted_cg(b, cfg1.shifts, fixed_iters=k)
        for s, beta in enumerate(cfg1.shifts):
            tr = o.true_residual(b, beta, res.W[s])
            assert abs(tr - res.res_est[s]) <= 1e-8 * max(tr, 1e-12) + 1e-13, (k, beta)
        assert np.all(np.diff(res.res_est) <= 1e-15)


def test_converged_solve_meets_tolerance(cfg1):
    o = oracle.from_problem(cfg1)
    b = o.rhs_canonical()
    res = o.shifted_cg(b, cfg1.shifts, tol=1e-10, max_iter=20000)
    assert res.status == 0
    for s, beta in enumerate(cfg1.shifts):
        assert res.res_est[s] < 1e-10
        assert o.true_residual(b, beta, res.W[s]) < 2e-10
    # larger shifts converge in no more iterations (Sec. 5.1, Table 6 discussion)
    assert np.all(np.diff(res.iters) <= 0)


# --------------------------------------------------------------------------
# Special cases and invariances
# --------------------------------------------------------------------------

def test_alpha_zero_ignores_unlabelled_rows(tiny):
    """alpha = 0: the Laplacian is off and only labelled rows enter B and b, so w is
    regularised LDA on the labelled rows (eq. 1): dropping unlabelled rows keeps w."""
    y = tiny.labels[0]
    o = oracle.from_problem(tiny, alpha=0.0)
    w = o.shifted_cg(o.rhs_canonical(), tiny.shifts, tol=1e-14, max_iter=5000).W
    keep = np.nonzero(y != 0)[0]
    cnt = np.diff(tiny.x_ptr)[keep]
    x_ptr = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    x_col = np.concatenate([tiny.x_col[tiny.x_ptr[i]:tiny.x_ptr[i + 1]] for i in keep])
    x_val = np.concatenate([tiny.x_val[tiny.x_ptr[i]:tiny.x_ptr[i + 1]] for i in keep])
    m = keep.size
    o2 = oracle.Oracle(x_ptr, x_col, x_val, np.zeros(m + 1, np.int64), np.zeros(0, np.int32),
                       np.zeros(0), y[keep], tiny.d, 0.0)
    w2 = o2.shifted_cg(o2.rhs_canonical(), tiny.shifts, tol=1e-14, max_iter=5000).W
    for s in range(len(tiny.shifts)):
        assert _rel(w2[s], w[s]) < 1e-10
    # and it is the ridge solution of the labelled total scatter
    X = oracle.dense_x(x_ptr, x_col, x_val, tiny.d)
    St, _ = oracle.dense_scatter_labelled(X, y[keep])
    b = o2.rhs_canonical()
    for s, beta in enumerate(tiny.shifts):
        assert _rel(w2[s], np.linalg.solve(St + beta * np.eye(tiny.d), b)) < 1e-9


def test_alpha_one_is_pure_manifold_term(tiny):
    """alpha = 1 (omega = 0): the labelled scatter drops out, B = X^T L X."""
    o = oracle.from_problem(tiny, alpha=1.0)
    X = _dense(tiny)
    XLX = oracle.dense_manifold(X, tiny.s_ptr, tiny.s_col, tiny.s_val)
    p = np.random.default_rng(4).standard_normal(tiny.d)
    assert _rel(o.apply(p), XLX @ p) < 1e-12


def test_large_shift_expansion(tiny):
    """(B + beta I)^{-1} b = b/beta - B b/beta^2 + O(beta^-3) for large beta."""
    o = oracle.from_problem(tiny)
    b = o.rhs_canonical()
    beta = 1e7
    w = o.shifted_cg(b, [beta], tol=1e-15, max_iter=100).W[0]
    approx = b / beta - o.apply(b) / beta ** 2
    assert _rel(w, approx) < 1e-6 * 10


def test_translation_invariance(tiny):
    """Centring (Sec. 2.5.2): X -> X + 1 t^T leaves B, d and w unchanged (graph fixed)."""
    X = _dense(tiny)
    t = np.random.default_rng(6).uniform(0.5, 2.0, size=tiny.d)
    n, d = X.shape
    full_ptr = (np.arange(n + 1) * d).astype(np.int64)
    full_col = np.tile(np.arange(d, dtype=np.int32), n)
    y = tiny.labels[0]
    o1 = oracle.Oracle(full_ptr, full_col, X.reshape(-1), tiny.s_ptr, tiny.s_col, tiny.s_val, y, d,
                       tiny.alpha)
    o2 = oracle.Oracle(full_ptr, full_col, (X + t).reshape(-1), tiny.s_ptr, tiny.s_col, tiny.s_val,
                       y, d, tiny.alpha)
    b1, b2 = o1.rhs_canonical(), o2.rhs_canonical()
    assert _rel(b2, b1) < 1e-12
    w1 = o1.shifted_cg(b1, tiny.shifts, tol=1e-14, max_iter=5000).W
    w2 = o2.shifted_cg(b2, tiny.shifts, tol=1e-14, max_iter=5000).W
    for s in range(len(tiny.shifts)):
        assert _rel(w2[s], w1[s]) < 1e-8


def test_linearity_in_rhs(cfg1):
    o = oracle.from_problem(cfg1)
    b = o.rhs_canonical()
    w1 = o.shifted_cg(b, cfg1.shifts, fixed_iters=20).W
    # scaling by a power of two is exact in every operation: bit-identical iterates
    w2 = o.shifted_cg(-4.0 * b, cfg1.shifts, fixed_iters=20).W
    assert np.array_equal(w2, -4.0 * w1)
    w3 = o.shifted_cg(3.0 * b, cfg1.shifts, fixed_iters=20).W
    assert _rel(w3, 3.0 * w1) < 1e-6      # rounding, amplified on the ill-conditioned shifts


def test_thread_count_does_not_change_results(cfg1):
    o = oracle.from_problem(cfg1)
    b = o.rhs_canonical()
    before = oracle.set_threads(1)
    w1 = o.shifted_cg(b, cfg1.shifts, fixed_iters=25).W
    oracle.set_threads(4)
    w4 = o.shifted_cg(b, cfg1.shifts, fixed_iters=25).W
    oracle.set_threads(before)
    assert np.array_equal(w1, w4)


# --------------------------------------------------------------------------
# Evaluation (Sec. 4: rating s = X w, AUC-ROC)
# --------------------------------------------------------------------------

def test_auc_rank_formula_equals_pairwise_bruteforce():
    rng = np.random.default_rng(7)
    for _ in range(5):
        s = np.round(rng.standard_normal(60), 1)        # ties on purpose
        y = np.where(rng.random(60) < 0.4, 1, -1)
        pos, neg = s[y > 0], s[y < 0]
        brute = ((pos[:, None] > neg[None, :]).sum() + 0.5 * (pos[:, None] == neg[None, :]).sum())
        brute /= pos.size * neg.size
        assert abs(oracle.auc(s, y) - brute) < 1e-15
    assert oracle.auc([3, 2, 1, 0], [1, 1, -1, -1]) == 1.0
    assert oracle.auc([0, 1, 2, 3], [1, 1, -1, -1]) == 0.0
    assert oracle.auc([1, 1, 1, 1], [1, -1, 1, -1]) == 0.5


def test_logistic_loss_closed_forms_and_gradient():
    """The held-out loss of the adjoint gradient (mean log(1 + e^{-y s})):
    log 2 at s = 0, vanishing for large margins, |y s| for large negative
    margins, element-wise brute force with math.log1p, and its gradient
    against central differences of the loss."""
    import math
    loss, g = oracle.logistic_loss(np.zeros(4), np.array([1, -1, 1, -1]))
    assert loss == math.log(2.0) and np.array_equal(g, np.array([-1, 1, -1, 1]) / 8.0)
    with np.errstate(over="ignore"):        # e^{800} in the gradient's denominator: the gradient is -0
        assert oracle.logistic_loss(np.array([800.0]), np.array([1]))[0] == 0.0
    assert oracle.logistic_loss(np.array([800.0]), np.array([-1]))[0] == 800.0
    rng = np.random.default_rng(9)
    s = rng.standard_normal(50) * 3.0
    y = np.where(rng.random(50) < 0.3, 1, -1)
    loss, g = oracle.logistic_loss(s, y)
    brute = sum(math.log1p(math.exp(-yi * si)) for si, yi in zip(s, y)) / s.size
    assert abs(loss - brute) < 1e-15 * max(1.0, brute)
    h = 1e-6
    for i in range(0, 50, 7):
        e = np.zeros(50)
        e[i] = h
        fd = (oracle.logistic_loss(s + e, y)[0] - oracle.logistic_loss(s - e, y)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-8, (i, fd, g[i])


def test_projection(tiny):
    o = oracle.from_problem(tiny)
    w = np.random.default_rng(8).standard_normal(tiny.d)
    assert _rel(o.project(w), _dense(tiny) @ w) < 1e-14


def test_planted_direction_is_found(cfg1):
    """Sanity of the method on the planted workload: the AUC of the rating over
    the 1,800 unlabelled rows is well above chance (0.5) for the best shift."""
    o = oracle.from_problem(cfg1)
    res = o.shifted_cg(o.rhs_canonical(), cfg1.shifts, tol=1e-8, max_iter=5000)
    unl = np.nonzero(cfg1.labels[0] == 0)[0]
    aucs = [oracle.auc(o.project(res.W[s])[unl], cfg1.truth[0][unl]) for s in range(len(cfg1.shifts))]
    assert max(aucs) > 0.65


# --------------------------------------------------------------------------
# Adjoint of the held-out loss (not in the paper; checks the library's adjoint)
# --------------------------------------------------------------------------

def test_dense_adjoint_gradient_equals_finite_differences(tiny):
    """d loss / d alpha and d loss / d beta from one adjoint solve equal central
    finite differences (h = 1e-4 on alpha and on log beta) of the loss itself."""
    X = _dense(tiny)
    y = tiny.labels[0]
    rows = tiny.heldout[0]
    yr = tiny.truth[0][rows]
    alpha, beta = 0.3, 0.05
    args = (X, tiny.s_ptr, tiny.s_col, tiny.s_val, y)
    loss, da, db, _ = oracle.adjoint_grad_dense(*args, alpha, beta, rows, yr)
    h = 1e-4
    lp = oracle.adjoint_grad_dense(*args, alpha + h, beta, rows, yr)[0]
    lm = oracle.adjoint_grad_dense(*args, alpha - h, beta, rows, yr)[0]
    assert abs((lp - lm) / (2 * h) - da) <= 1e-6 * max(1.0, abs(da))
    lp = oracle.adjoint_grad_dense(*args, alpha, beta * np.exp(h), rows, yr)[0]
    lm = oracle.adjoint_grad_dense(*args, alpha, beta * np.exp(-h), rows, yr)[0]
    # d/d(log beta) = beta d/d beta
    assert abs((lp - lm) / (2 * h) - beta * db) <= 1e-6 * max(1.0, abs(beta * db))


def test_sparse_adjoint_equals_dense_adjoint(tiny):
    """The sparse adjoint gradient (C oracle CG, sparse products) equals the dense
    one (explicit B, direct solves) at two points and in the finite differences
    of its own loss; a dropped S_t term in dB/dalpha fails the alpha check."""
    X = _dense(tiny)
    y = tiny.labels[0]
    rows = tiny.heldout[0]
    yr = tiny.truth[0][rows]
    for alpha, beta in ((0.3, 0.05), (0.7, 2.0)):
        o = oracle.from_problem(tiny, alpha=alpha)
        ls, das, dbs, ws = oracle.adjoint_grad_sparse(o, tiny.x_ptr, tiny.x_col, tiny.x_val, tiny.s_ptr,
                                                      tiny.s_col, tiny.s_val, rows, yr, beta, tol=1e-14)
        ld, dad, dbd, wd = oracle.adjoint_grad_dense(X, tiny.s_ptr, tiny.s_col, tiny.s_val, y, alpha, beta, rows, yr)
        assert np.linalg.norm(ws - wd) <= 1e-10 * np.linalg.norm(wd)
        assert abs(ls - ld) <= 1e-12 * abs(ld)
        assert abs(das - dad) <= 1e-8 * abs(dad) and abs(dbs - dbd) <= 1e-8 * abs(dbd)
    # a plausible mistake, dB/dalpha = X^T L X (dropping the -S_t^l of omega = 1 - alpha),
    # moves the alpha derivative far beyond the agreement asserted above
    St, mu = oracle.dense_scatter_labelled(X, y)
    XLX = oracle.dense_manifold(X, tiny.s_ptr, tiny.s_col, tiny.s_val)
    A = (1 - alpha) * St + alpha * XLX + beta * np.eye(X.shape[1])
    _, g = oracle.logistic_loss((X[rows] - mu) @ wd, yr)
    lam = np.linalg.solve(A, (X[rows] - mu).T @ g)
    assert abs(-lam @ (XLX @ wd) - dad) > 1e-3 * abs(dad)


def test_regression_operator_is_xtx():
    """CSR-SDA's regression step (Algorithm 5, line 5): the oracle's regression
    operator is X^T X + sigma I, and its shifted CG reaches the dense solutions
    of (X^T X + beta I) w = X^T z."""
    p = synth.custom_problem(150, 40, 7, seed=13, values="counts", shifts=(1e-1, 1e1, 3))
    o = oracle.Oracle.regression(p.x_ptr, p.x_col, p.x_val, p.d)
    X = oracle.dense_x(p.x_ptr, p.x_col, p.x_val, p.d)
    x = np.random.default_rng(2).standard_normal(p.d)
    assert np.linalg.norm(o.apply(x, 0.3) - (X.T @ (X @ x) + 0.3 * x)) < 1e-10 * np.linalg.norm(x) * np.linalg.norm(X) ** 2
    z = np.random.default_rng(4).uniform(-1.0, 1.0, p.n)
    b = X.T @ z
    res = o.shifted_cg(b, p.shifts, tol=1e-13, max_iter=5000)
    for s, beta in enumerate(p.shifts):
        w = np.linalg.solve(X.T @ X + beta * np.eye(p.d), b)
        assert np.linalg.norm(res.W[s] - w) < 1e-9 * np.linalg.norm(w)


def _identity_x(n):
    return np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n)


def test_sa_sda_operator_with_identity_data():
    """SA-SDA (Algorithm 6) is the SDA operator with X = I_N: the oracle's
    paper form (I - 1_l 1^T / l) M equals the symmetric M - omega 1_l 1_l^T / l
    (M 1 = omega 1_l), and its canonical direction d = 1_+/N+ - 1_-/N- is
    parallel to Algorithm 6's [W 0; 0 0] r for r orthogonal to 1_l."""
    p = synth.custom_problem(180, 30, 6, seed=17, values="binary", n_labelled=60, k=5)
    n, y, a = p.n, p.labels[0], p.alpha
    om = 1.0 - a
    xp, xc, xv = _identity_x(n)
    o = oracle.Oracle(xp, xc, xv, p.s_ptr, p.s_col, p.s_val, y, n, a)
    Sd = np.zeros((n, n))
    for i in range(n):
        Sd[i, p.s_col[p.s_ptr[i]:p.s_ptr[i + 1]]] = p.s_val[p.s_ptr[i]:p.s_ptr[i + 1]]
    L = np.diag(Sd.sum(1)) - Sd
    one_l = (y != 0).astype(float)
    ell = one_l.sum()
    Mt = om * np.diag(one_l) + a * L - om * np.outer(one_l, one_l) / ell
    x = np.random.default_rng(5).standard_normal(n)
    assert np.linalg.norm(o.apply(x, 0.2) - (Mt @ x + 0.2 * x)) < 1e-12 * np.linalg.norm(x) * max(1.0, np.abs(Mt).max())
    pos, neg = (y > 0).astype(float), (y < 0).astype(float)
    r = np.random.default_rng(6).uniform(-1.0, 1.0, n)
    r = r - (one_l @ r) / ell                  # Algorithm 6, orthogonalisation: r - 1 <1_l, r> / l
    Wr = pos * (pos @ r) / pos.sum() + neg * (neg @ r) / neg.sum()
    d = o.rhs_canonical()
    assert np.linalg.norm(Wr - (pos @ r) * d) < 1e-12 * np.linalg.norm(Wr)
    res = o.shifted_cg(d, p.shifts, tol=1e-13, max_iter=5000)
    for s, beta in enumerate(p.shifts):
        z = np.linalg.solve(Mt + beta * np.eye(n), d)
        assert np.linalg.norm(res.W[s] - z) < 1e-9 * np.linalg.norm(z)


# --------------------------------------------------------------------------
# Similarity graph (Sec. 2.4; Tanimoto, Sec. 5.1)
# --------------------------------------------------------------------------

def _knn_by_sets(x_ptr, x_col, k, cap=None, threshold=0.0):
    """The definition with Python sets and a double loop."""
    n = x_ptr.size - 1
    rows = [set(x_col[x_ptr[i]:x_ptr[i + 1]].tolist()) for i in range(n)]
    cnt = {}
    for r in rows:
        for f in r:
            cnt[f] = cnt.get(f, 0) + 1
    edges = {}
    for i in range(n):
        best = []
        for j in range(n):
            if j == i:
                continue
            shared = rows[i] & rows[j]
            if cap is not None:
                if not any(cnt[f] <= cap for f in shared):
                    continue
            if not shared:
                continue
            s = len(shared) / len(rows[i] | rows[j])
            if s < threshold:
                continue
            best.append((-s, j, s))
        best.sort()
        for _, j, s in best[:k]:
            edges[(i, j)] = s
            edges[(j, i)] = s
    return edges


@pytest.mark.parametrize("cap,thr", [(None, 0.0), (3, 0.0), (None, 0.25)])
def test_knn_graph_oracle_equals_set_definition(cap, thr):
    from paper_1709_04794_gb300 import synth
    p = synth.custom_problem(90, 40, 6, seed=13, n_labelled=20, k=3)
    rp, col, val = oracle.knn_graph(p.x_ptr, p.x_col, p.d, 4, cap=cap, threshold=thr)
    ref = _knn_by_sets(p.x_ptr, p.x_col, 4, cap=cap, threshold=thr)
    got = {(i, int(col[e])): float(val[e]) for i in range(p.n) for e in range(rp[i], rp[i + 1])}
    assert got.keys() == ref.keys() and all(got[key] == ref[key] for key in ref)
    assert all(i != j for (i, j) in got) and all((j, i) in got for (i, j) in got)
    assert all(0.0 < v <= 1.0 for v in got.values())


def test_knn_graph_oracle_equals_input_generator():
    """Two independent implementations of the same definition: the oracle's
    dense one and the input generator's candidate lists in C."""
    from paper_1709_04794_gb300 import synth
    p = synth.custom_problem(400, 150, 9, seed=17, n_labelled=40, k=5)
    for cap in (None, 12):
        nbr, sim = synth.knn_lists(p.x_ptr, p.x_col, p.d, 5, cap)
        g_rp, g_col, g_val = synth.union_graph(nbr, sim)
        o_rp, o_col, o_val = oracle.knn_graph(p.x_ptr, p.x_col, p.d, 5, cap=cap)
        assert np.array_equal(g_rp, o_rp) and np.array_equal(g_col, o_col) and np.array_equal(g_val, o_val)


def test_fixed_run_ends_at_a_vanished_residual(tiny):
    """Algorithms 2 and 3 iterate while a residual remains: a fixed-iteration
    run at a shift far above ||B|| converges until <r, r> underflows to exactly
    zero and ends there (no breakdown on <p, q> = 0), with the exact solution,
    i.e. the dense solve's."""
    o = oracle.from_problem(tiny)
    b = o.rhs_canonical()
    beta = 1e5
    X = oracle.dense_x(tiny.x_ptr, tiny.x_col, tiny.x_val, tiny.d)
    B = oracle.dense_operator(X, tiny.s_ptr, tiny.s_col, tiny.s_val, tiny.labels[0], tiny.alpha)
    w, it, res, rc = o.cg(b, beta, fixed_iters=2000)
    assert rc == 0 and it < 2000, (rc, it)
    sh = o.shifted_cg(b, [beta, 2 * beta], fixed_iters=2000)
    assert sh.status == 0 and sh.total_iters < 2000, (sh.status, sh.total_iters)
    for s, bt in enumerate((beta, 2 * beta)):
        ref = np.linalg.solve(B + bt * np.eye(tiny.d), b)
        assert np.linalg.norm(sh.W[s] - ref) <= 1e-13 * np.linalg.norm(ref), s
    ref = np.linalg.solve(B + beta * np.eye(tiny.d), b)
    assert np.linalg.norm(w - ref) <= 1e-13 * np.linalg.norm(ref)
