"""FP64 CPU oracle for fast binary SDA -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, the smoke check and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA library: the
iterative solver is plain C (``sda_oracle.c``, Algorithms 2, 3 and 7), and
the dense checks below are NumPy written from the paper's definitions.

Functions and what they follow:

* :class:`Oracle`            - the C oracle: mu_l (Alg. 7 step 3), the
  operator in the paper's form (Alg. 7 step 4, Sec. 3.2.3), the RHS of
  Alg. 7 step 4, CG (Alg. 2), shifted CG (Alg. 3), s = X w (Sec. 4);
  ``Oracle.regression``: B = X^T X of CSR-SDA's regression step (Alg. 5,
  line 5).
* :func:`dense_scatter_labelled` - S_t^l = sum_{i in l} (x_i - mu_l)(x_i - mu_l)^T
  (total labelled scatter, eq. 7 with centring of Sec. 2.5.2).
* :func:`dense_manifold`     - X^T L X from the regulariser
  R(w) = sum_ij s_ij (w^T x_i - w^T x_j)^2 = 2 w^T X^T L X w (Sec. 2.3).
* :func:`dense_between`      - labelled between-class scatter
  sum_c N_c (mu_c - mu_l)(mu_c - mu_l)^T (left side of eq. 7, centred).
* :func:`auc`                - AUC-ROC of the rating s = X w (Sec. 4), by the
  rank-sum formula with average ranks for ties.
* :func:`adjoint_grad_dense` - d loss / d(alpha, beta) by the adjoint of the
  regularised system (not in the paper; checks the library's adjoint).
* :func:`adjoint_grad_sparse` - the same through the C oracle's CG and sparse
  products, for problems too large to densify.
* :func:`knn_graph`          - the similarity graph of Sec. 2.4 (Tanimoto kNN,
  union of the directed lists) from dense binary supports, small inputs.

Every function above is pinned by the ``-m "not gpu"`` tests against
closed forms, dense definitions, special cases and brute force
(tests/test_oracle_pins.py), and tests/test_oracle_mutations.py plants
plausible mistakes in copies of the C oracle to show the pins catch them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "sda_oracle.c")
_SO = os.path.join(_DIR, "_sda_oracle.so")

_i64p = ctypes.c_void_p


def build(force: bool = False, extra_flags: tuple = (), out: str | None = None) -> str:
    """Compile the C oracle in place (gcc, OpenMP, strict IEEE FP64)."""
    import platform
    out = out or _SO
    stamp = out + ".arch"
    stale = (not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC)
             or not os.path.exists(stamp) or open(stamp).read().strip() != platform.machine())
    if force or extra_flags or stale:
        tmp = out + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", *extra_flags, _SRC,
               "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
        os.replace(tmp, out)
        with open(stamp, "w") as f:
            f.write(platform.machine() + "\n")
    return out


def _load(path: str):
    lib = ctypes.CDLL(path)
    vp, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.oracle_create.restype = vp
    lib.oracle_create.argtypes = [i64, i64, vp, vp, vp, vp, vp, vp, vp, f64, f64]
    lib.oracle_create_regression.restype = vp
    lib.oracle_create_regression.argtypes = [i64, i64, vp, vp, vp, vp, vp]
    lib.oracle_destroy.argtypes = [vp]
    lib.oracle_destroy.restype = None
    lib.oracle_set_threads.argtypes = [i32]
    lib.oracle_set_threads.restype = i32
    lib.oracle_class_means.argtypes = [vp, vp, vp, vp, vp]
    lib.oracle_class_means.restype = None
    lib.oracle_apply.argtypes = [vp, f64, vp, vp]
    lib.oracle_apply.restype = None
    lib.oracle_rhs_from_r.argtypes = [vp, vp, vp]
    lib.oracle_rhs_from_r.restype = None
    lib.oracle_project.argtypes = [vp, vp, vp]
    lib.oracle_project.restype = None
    lib.oracle_cg.argtypes = [vp, vp, f64, f64, i32, i32, vp, vp, vp]
    lib.oracle_cg.restype = i32
    lib.oracle_shifted_cg.argtypes = [vp, vp, vp, i32, f64, i32, i32, vp, vp, vp, vp]
    lib.oracle_shifted_cg.restype = i32
    return lib


_LIB = {}


def lib(path: str | None = None):
    path = path or build()
    if path not in _LIB:
        _LIB[path] = _load(path)
    return _LIB[path]


def set_threads(t: int) -> int:
    return lib().oracle_set_threads(int(t))


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


@dataclass
class ShiftedResult:
    W: np.ndarray          # [S, D]
    iters: np.ndarray      # [S]
    res_est: np.ndarray    # [S]
    total_iters: int
    status: int


class Oracle:
    """One (X, S, labels, alpha, omega) problem held by the C oracle."""

    def __init__(self, x_ptr, x_col, x_val, s_ptr, s_col, s_val, y, d, alpha, omega=None,
                 so_path: str | None = None):
        self._lib = lib(so_path)
        self.n = int(np.asarray(x_ptr).size - 1)
        self.d = int(d)
        self._keep = [_c(x_ptr, np.int64), _c(x_col, np.int32), _c(x_val, np.float64),
                      _c(s_ptr, np.int64), _c(s_col, np.int32), _c(s_val, np.float64),
                      _c(y, np.int8)]
        self.alpha = float(alpha)
        self.omega = float(1.0 - alpha if omega is None else omega)
        self._h = self._lib.oracle_create(self.n, self.d, *(a.ctypes.data for a in self._keep),
                                          self.alpha, self.omega)
        if not self._h:
            raise ValueError("oracle_create failed (allocation or column index out of range)")

    @classmethod
    def regression(cls, x_ptr, x_col, x_val, d, so_path: str | None = None):
        """B = X^T X, the operator of CSR-SDA's regression step (Algorithm 5, line 5)."""
        self = cls.__new__(cls)
        self._lib = lib(so_path)
        self.n = int(np.asarray(x_ptr).size - 1)
        self.d = int(d)
        self._keep = [_c(x_ptr, np.int64), _c(x_col, np.int32), _c(x_val, np.float64),
                      np.zeros(self.n + 1, np.int64), np.ones(self.n, np.int8)]
        self.alpha, self.omega = 0.0, 1.0
        self._h = self._lib.oracle_create_regression(self.n, self.d, *(a.ctypes.data for a in self._keep))
        if not self._h:
            raise ValueError("oracle_create_regression failed (allocation or column index out of range)")
        return self

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_destroy(h)
            self._h = None

    # -- Alg. 7 step 3 and the class means ---------------------------------
    def class_means(self):
        d = self.d
        mu, mp, mn, cnt = np.empty(d), np.empty(d), np.empty(d), np.empty(3)
        self._lib.oracle_class_means(self._h, mu.ctypes.data, mp.ctypes.data, mn.ctypes.data,
                                     cnt.ctypes.data)
        return mu, mp, mn, cnt

    def rhs_canonical(self):
        """b = d = mu_+ - mu_- (the direction of the rank-1 right-hand side)."""
        _, mp, mn, _ = self.class_means()
        return mp - mn

    def rhs_from_r(self, r):
        r = _c(r, np.float64)
        b = np.empty(self.d)
        self._lib.oracle_rhs_from_r(self._h, r.ctypes.data, b.ctypes.data)
        return b

    # -- operator -----------------------------------------------------------
    def apply(self, p, sigma: float = 0.0):
        p = _c(p, np.float64)
        q = np.empty(self.d)
        self._lib.oracle_apply(self._h, float(sigma), p.ctypes.data, q.ctypes.data)
        return q

    def project(self, w):
        w = _c(w, np.float64)
        s = np.empty(self.n)
        self._lib.oracle_project(self._h, w.ctypes.data, s.ctypes.data)
        return s

    # -- solvers -----------------------------------------------------------
    def cg(self, b, beta, tol=1e-12, max_iter=10000, fixed_iters=0):
        b = _c(b, np.float64)
        w = np.empty(self.d)
        it, res = ctypes.c_int(), ctypes.c_double()
        rc = self._lib.oracle_cg(self._h, b.ctypes.data, float(beta), float(tol), int(max_iter),
                                 int(fixed_iters), w.ctypes.data, ctypes.byref(it), ctypes.byref(res))
        return w, it.value, res.value, rc

    def shifted_cg(self, b, betas, tol=1e-12, max_iter=10000, fixed_iters=0) -> ShiftedResult:
        b = _c(b, np.float64)
        betas = _c(betas, np.float64)
        ns = betas.size
        W = np.empty((ns, self.d))
        iters = np.zeros(ns, dtype=np.int32)
        res = np.zeros(ns)
        tot = ctypes.c_int()
        rc = self._lib.oracle_shifted_cg(self._h, b.ctypes.data, betas.ctypes.data, ns, float(tol),
                                         int(max_iter), int(fixed_iters), W.ctypes.data,
                                         iters.ctypes.data, res.ctypes.data, ctypes.byref(tot))
        return ShiftedResult(W, iters, res, tot.value, rc)

    def true_residual(self, b, beta, w):
        """||b - (B + beta I) w|| / ||b|| in FP64."""
        r = b - self.apply(w, beta)
        nb = np.linalg.norm(b)
        return float(np.linalg.norm(r) / nb) if nb > 0 else float(np.linalg.norm(r))


def from_problem(prob, target: int = 0, alpha: float | None = None, omega: float | None = None,
                 so_path: str | None = None) -> Oracle:
    a = prob.alpha if alpha is None else alpha
    return Oracle(prob.x_ptr, prob.x_col, prob.x_val, prob.s_ptr, prob.s_col, prob.s_val,
                  prob.labels[target], prob.d, a, omega, so_path)


# ---------------------------------------------------------------------------
# Dense definitions (tiny inputs only)
# ---------------------------------------------------------------------------


def dense_x(x_ptr, x_col, x_val, d):
    n = x_ptr.size - 1
    X = np.zeros((n, d))
    row = np.repeat(np.arange(n), np.diff(x_ptr))
    X[row, x_col] = x_val
    return X


def dense_scatter_labelled(X, y):
    """S_t^l = sum over labelled samples of (x_i - mu_l)(x_i - mu_l)^T."""
    lab = np.nonzero(y != 0)[0]
    mu = X[lab].mean(axis=0)
    C = X[lab] - mu
    return C.T @ C, mu


def dense_manifold(X, s_ptr, s_col, s_val):
    """X^T L X = 1/2 sum_(i,j) s_ij (x_i - x_j)(x_i - x_j)^T over the stored (ordered) pairs."""
    n = s_ptr.size - 1
    src = np.repeat(np.arange(n), np.diff(s_ptr))
    Dl = X[src] - X[s_col]
    return 0.5 * (Dl * s_val[:, None]).T @ Dl


def dense_between(X, y):
    """sum_c N_c (mu_c - mu_l)(mu_c - mu_l)^T over the two labelled classes."""
    lab = y != 0
    mu = X[lab].mean(axis=0)
    out = np.zeros((X.shape[1], X.shape[1]))
    for c in (1, -1):
        m = y == c
        dc = X[m].mean(axis=0) - mu
        out += m.sum() * np.outer(dc, dc)
    return out


def dense_operator(X, s_ptr, s_col, s_val, y, alpha, omega=None):
    omega = 1.0 - alpha if omega is None else omega
    St, _ = dense_scatter_labelled(X, y)
    return omega * St + alpha * dense_manifold(X, s_ptr, s_col, s_val)


def auc(scores, truth):
    """AUC-ROC by the rank-sum (Mann-Whitney) formula, average ranks for ties."""
    scores = np.asarray(scores, dtype=np.float64)
    truth = np.asarray(truth)
    pos = truth > 0
    n_pos, n_neg = int(pos.sum()), int((~pos).sum())
    if n_pos == 0 or n_neg == 0:
        return float("nan")
    order = np.argsort(scores, kind="mergesort")
    s_sorted = scores[order]
    ranks = np.empty(scores.size)
    i = 0
    while i < s_sorted.size:
        j = i
        while j + 1 < s_sorted.size and s_sorted[j + 1] == s_sorted[i]:
            j += 1
        ranks[order[i:j + 1]] = 0.5 * (i + j) + 1.0
        i = j + 1
    return float((ranks[pos].sum() - n_pos * (n_pos + 1) / 2.0) / (n_pos * n_neg))


def logistic_loss(s, y):
    """mean log(1 + exp(-y s)) and its derivative with respect to s."""
    z = -np.asarray(y, dtype=np.float64) * s
    loss = np.mean(np.logaddexp(0.0, z))
    g = -np.asarray(y, dtype=np.float64) / (1.0 + np.exp(-z)) / s.size
    return float(loss), g


def adjoint_grad_dense(X, s_ptr, s_col, s_val, y, alpha, beta, rows, y_rows, b=None):
    """Dense d loss/d alpha and d loss/d beta of the held-out logistic loss.

    w = (B(alpha) + beta I)^{-1} b with B = (1 - alpha) S_t^l + alpha X^T L X,
    s_h = (X_h - 1 mu_l^T) w, loss = mean log(1 + exp(-y_h s_h)).
    """
    St, mu = dense_scatter_labelled(X, y)
    XLX = dense_manifold(X, s_ptr, s_col, s_val)
    if b is None:
        b = X[y > 0].mean(axis=0) - X[y < 0].mean(axis=0)
    A = (1.0 - alpha) * St + alpha * XLX + beta * np.eye(X.shape[1])
    w = np.linalg.solve(A, b)
    Xh = X[rows] - mu
    s = Xh @ w
    loss, g = logistic_loss(s, y_rows)
    lam = np.linalg.solve(A, Xh.T @ g)
    d_beta = -lam @ w
    d_alpha = -lam @ ((XLX - St) @ w)
    return loss, float(d_alpha), float(d_beta), w


def adjoint_grad_sparse(o: Oracle, x_ptr, x_col, x_val, s_ptr, s_col, s_val, rows, y_rows, beta,
                        tol=1e-12, max_iter=100000, fixed_iters=0, w=None):
    """d loss/d alpha and d loss/d beta of the held-out logistic loss, for
    problems too large for adjoint_grad_dense: the two solves are the C
    oracle's CG (Algorithm 2) on its operator, the products sparse.

    w = (B + beta I)^{-1} d, s_h = (X_h - 1 mu_l^T) w, loss = mean log(1 + exp(-y s_h));
    lambda = (B + beta I)^{-1} (X_h - 1 mu_l^T)^T g,  g = d loss / d s_h;
    d loss/d beta = -lambda^T w,  d loss/d alpha = -lambda^T (dB/dalpha) w with
    dB/dalpha = X^T L X - S_t^l (B = (1 - alpha) S_t^l + alpha X^T L X, eq. 7).
    fixed_iters > 0 runs both CG solves for exactly that many iterations (the
    fixed-iteration protocol of Sec. 5.2); a given w skips the forward solve.
    Returns (loss, d_alpha, d_beta, w)."""
    import scipy.sparse as sp
    n, d = o.n, o.d
    X = sp.csr_matrix((np.asarray(x_val, float), np.asarray(x_col), np.asarray(x_ptr)), shape=(n, d))
    S = sp.csr_matrix((np.asarray(s_val, float), np.asarray(s_col), np.asarray(s_ptr)), shape=(n, n))
    L = sp.diags(np.asarray(S.sum(axis=1)).ravel()) - S
    mu, mp, mn, _ = o.class_means()
    lab = (np.asarray(o._keep[6]) != 0).astype(float)
    if w is None:
        w, _, _, rc = o.cg(mp - mn, beta, tol=tol, max_iter=max_iter, fixed_iters=fixed_iters)
    rows = np.asarray(rows)
    s = X[rows] @ w - mu @ w
    loss, g = logistic_loss(s, y_rows)
    c = X[rows].T @ g - mu * g.sum()
    lam, _, _, rc2 = o.cg(c, beta, tol=tol, max_iter=max_iter, fixed_iters=fixed_iters)
    u = X @ w - mu @ w                      # centred ratings of every sample
    St_w = X.T @ (lab * u) - mu * (lab * u).sum()
    XLX_w = X.T @ (L @ (X @ w))
    return loss, float(-lam @ (XLX_w - St_w)), float(-lam @ w), w


def knn_graph(x_ptr, x_col, d, k, cap=None, threshold=0.0):
    """The similarity graph of Sec. 2.4 by its definition (small inputs):
    s_ij = |x_i and x_j| / |x_i or x_j| on the binary supports (Tanimoto,
    Sec. 5.1); row i's candidates are the rows j != i sharing a feature (only
    features of column count <= cap when cap is given); its k nearest are the
    candidates of positive similarity (and >= threshold) ranked by (similarity
    descending, row index ascending); the edges are the union of the directed
    lists.  Returns the CSR (row_ptr int64, col int32, val float64), rows sorted."""
    n = np.asarray(x_ptr).size - 1
    B = np.zeros((n, d), dtype=np.int64)
    row = np.repeat(np.arange(n), np.diff(x_ptr))
    B[row, np.asarray(x_col)] = 1
    inter = B @ B.T
    size = B.sum(axis=1)
    union = size[:, None] + size[None, :] - inter
    jac = np.where(inter > 0, inter / np.maximum(union, 1), 0.0)
    if cap is None:
        cand = inter > 0
    else:
        R = B[:, B.sum(axis=0) <= cap]
        cand = (R @ R.T) > 0
    np.fill_diagonal(cand, False)
    edges = {}
    for i in range(n):
        js = np.nonzero(cand[i] & (jac[i] > 0) & (jac[i] >= threshold))[0]
        order = sorted(js.tolist(), key=lambda j: (-jac[i, j], j))[:k]
        for j in order:
            edges[(i, j)] = jac[i, j]
            edges[(j, i)] = jac[i, j]
    keys = sorted(edges)
    rp = np.zeros(n + 1, dtype=np.int64)
    for (i, _) in keys:
        rp[i + 1] += 1
    rp = np.cumsum(rp)
    col = np.array([j for (_, j) in keys], dtype=np.int32)
    val = np.array([edges[key] for key in keys], dtype=np.float64)
    return rp, col, val
