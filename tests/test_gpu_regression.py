"""The regression step of CSR-SDA (Algorithm 5, line 5): shifted CG on
(X^T X + beta I) w = X^T z through sda_build_regression, against the FP64
oracle's regression operator (Oracle.regression, pinned to dense solves in
test_oracle_pins.py).

Bars: apply 1e-12 relative (FP64); FP64 iterates after 3 fixed iterations
1e-9, after 9 1e-6 (worse conditioned than the SDA operator); converged FP64
(tol 1e-10) 1e-6 on
w with FP64 true residuals below 1e-9; the FP16 path's true residual within
20 x tol; projection = X w; misuse rejected.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_04794_gb300 import sda, synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def reg():
    """4,000 x 1,500 count features (ragged tiles, split head columns), z ~ U(-1, 1)."""
    p = synth.custom_problem(4001, 1499, 18, seed=29, values="counts", shifts=(1e-2, 1e2, 6))
    z = np.random.default_rng(7).uniform(-1.0, 1.0, p.n)
    rows = np.repeat(np.arange(p.n), np.diff(p.x_ptr))
    b = np.bincount(p.x_col, weights=p.x_val * z[rows], minlength=p.d)   # X^T z
    o = oracle.Oracle.regression(p.x_ptr, p.x_col, p.x_val, p.d)
    return p, b, o


def _op(p, compute):
    return sda.Operator.regression(p.x_ptr, p.x_col, p.x_val, p.d, compute=compute)


def _solve(op, p, b, tol=1e-10, fixed=0, check=1):
    ns = len(p.shifts)
    w = torch.empty((1, ns, p.d), dtype=torch.float64, device="cuda")
    o = sda.sda_default_opts()
    o.tol, o.max_iter, o.fixed_iters, o.check_residual = tol, 20000, fixed, check
    o.rhs_mode = sda.SDA_RHS_GIVEN
    code, rep = sda.sda_solve_shifts(op.handle, p.shifts, o, w_out=w, n_report=1, rhs=b[None, :])
    return code, rep[0], w[0].cpu().numpy()


def test_regression_apply(reg):
    p, b, o = reg
    op = _op(p, "f64")
    x = np.random.default_rng(1).standard_normal(p.d)
    q = torch.empty(p.d, dtype=torch.float64, device="cuda")
    sda.sda_operator_apply(op.handle, 0, 0.5, torch.from_numpy(x).cuda(), q)
    assert _rel(q.cpu().numpy(), o.apply(x, 0.5)) < 1e-12


@pytest.mark.parametrize("k,bar", [(3, 1e-9), (9, 1e-6)])
def test_regression_fixed_iterations(reg, k, bar):
    """X^T X of count data is far worse conditioned than the SDA operator
    (kappa ~ 1e8 at beta = 1e-2), so the summation-order rounding of the two
    sides grows faster with k: 1e-9 holds for the first iterations, 1e-6 at 9
    (measured 6.6e-8)."""
    p, b, o = reg
    code, rep, w = _solve(_op(p, "f64"), p, b, fixed=k, check=0)
    ref = o.shifted_cg(b, p.shifts, fixed_iters=k)
    for s in range(len(p.shifts)):
        assert _rel(w[s], ref.W[s]) < bar, (s, _rel(w[s], ref.W[s]))


def test_regression_converged(reg):
    p, b, o = reg
    code, rep, w = _solve(_op(p, "f64"), p, b, tol=1e-10)
    assert code == sda.SDA_OK
    ref = o.shifted_cg(b, p.shifts, tol=1e-12, max_iter=50000)
    for s in range(len(p.shifts)):
        assert _rel(w[s], ref.W[s]) < 1e-6, s
        assert rep[s]["true_residual"] < 1e-9, rep[s]


def test_regression_mixed(reg):
    p, b, o = reg
    tol = 1e-6
    code, rep, w = _solve(_op(p, "f16"), p, b, tol=tol)
    assert code == sda.SDA_OK
    for s, beta in enumerate(p.shifts):
        assert o.true_residual(b, beta, w[s]) < 20 * tol, s


def test_regression_projection(reg):
    p, b, o = reg
    op = _op(p, "f64")
    code, rep, w = _solve(op, p, b, fixed=5, check=0)
    ns = len(p.shifts)
    scores = torch.empty((ns, p.n), dtype=torch.float64, device="cuda")
    sda.sda_project(op.handle, torch.from_numpy(w).cuda(), ns, scores, 1, 0)
    X = oracle.dense_x(p.x_ptr, p.x_col, p.x_val, p.d)
    assert _rel(scores.cpu().numpy(), w @ X.T) < 1e-12


def test_regression_rejects_misuse(reg):
    p, b, o = reg
    op = _op(p, "f64")
    w = torch.empty((1, len(p.shifts), p.d), dtype=torch.float64, device="cuda")
    o2 = sda.sda_default_opts()          # canonical right-hand side: undefined here
    with pytest.raises(sda.SDAError) as e:
        sda.sda_solve_shifts(op.handle, p.shifts, o2, w_out=w, n_report=1)
    assert e.value.code == sda.SDA_ERR_INVALID_ARG
    o3 = sda.sda_default_opts()
    o3.rhs_mode, o3.alpha = sda.SDA_RHS_GIVEN, 0.5
    with pytest.raises(sda.SDAError) as e:
        sda.sda_solve_shifts(op.handle, p.shifts, o3, w_out=w, n_report=1, rhs=b[None, :])
    assert e.value.code == sda.SDA_ERR_INVALID_ARG
