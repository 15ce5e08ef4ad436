"""Stored expected values (tests/golden/small_300x96_fp64.json and
small_300x96_modes_fp64.json, written by tests/golden/make_golden.py from the
FP64 oracle): a 300 x 96 count problem, one target, four shifts 1e-1..1e2,
under the SDA operator, CSR-SDA's regression operator and SA-SDA's operator.

CPU: the oracle still reproduces the stored solutions (bit for bit up to
1e-12) and they solve the dense definition (B + beta I) w = d of eq. 7 /
Sec. 3.2.3 to 1e-9.  GPU: the CUDA FP64 path matches the stored solutions to
1e-9 relative (kappa <= 1e3 on these shifts, both sides converged to 1e-12)
and the stored AUCs to 4 decimals; the mixed FP16 path reaches 20 x tol in FP64
true residual.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1709_04794_gb300 import synth

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "small_300x96_fp64.json")


@pytest.fixture(scope="module")
def golden():
    g = json.load(open(PATH))
    wl = synth.Workload(name="golden", n=g["n"], d=g["d"], nnz_mean=10, values="counts", n_targets=1,
                        labelled=("fixed", 80), pos_frac=("fixed", 0.3), knn_k=5, alpha=g["alpha"],
                        shifts=(1e-1, 1e2, 4), seed=1709, value_dtype="f64")
    p = synth.Problem(wl, np.asarray(g["x_ptr"], np.int64), np.asarray(g["x_col"], np.int32),
                      np.asarray(g["x_val"], np.float64), np.asarray(g["s_ptr"], np.int64),
                      np.asarray(g["s_col"], np.int32), np.asarray(g["s_val"], np.float64),
                      np.asarray([g["labels"]], np.int8), np.asarray([g["truth"]], np.int8),
                      [np.asarray(g["heldout"], np.int64)], np.asarray(g["shifts"]), g["alpha"])
    return p, g


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_golden_oracle_reproduces(golden):
    p, g = golden
    o = oracle.from_problem(p)
    b = o.rhs_canonical()
    assert np.array_equal(b, np.asarray(g["rhs"]))
    res = o.shifted_cg(b, p.shifts, tol=1e-13, max_iter=50000)
    W = np.asarray(g["w"])
    for s in range(len(p.shifts)):
        assert _rel(res.W[s], W[s]) < 1e-12, s
    assert res.iters.tolist() == g["iters"]


def test_golden_solves_dense_definition(golden):
    p, g = golden
    X = oracle.dense_x(p.x_ptr, p.x_col, p.x_val, p.d)
    B = oracle.dense_operator(X, p.s_ptr, p.s_col, p.s_val, p.labels[0], p.alpha)
    b = np.asarray(g["rhs"])
    for s, beta in enumerate(p.shifts):
        w = np.linalg.solve(B + beta * np.eye(p.d), b)
        assert _rel(np.asarray(g["w"][s]), w) < 1e-9, s


@pytest.mark.gpu
def test_golden_gpu_fp64(golden):
    import torch
    from paper_1709_04794_gb300 import sda
    p, g = golden
    op = sda.Operator(p, compute="f64")
    ns = len(p.shifts)
    w = torch.empty((1, ns, p.d), dtype=torch.float64, device="cuda")
    o = sda.sda_default_opts()
    o.tol, o.max_iter = 1e-12, 20000
    code, rep = sda.sda_solve_shifts(op.handle, p.shifts, o, w_out=w, n_report=1)
    assert code == sda.SDA_OK
    W = w[0].cpu().numpy()
    X = oracle.dense_x(p.x_ptr, p.x_col, p.x_val, p.d)
    rows = np.asarray(g["heldout"])
    for s in range(ns):
        assert _rel(W[s], np.asarray(g["w"][s])) < 1e-9, s
        assert abs(oracle.auc(X[rows] @ W[s], p.truth[0][rows]) - g["auc"][s]) < 5e-5


@pytest.mark.gpu
def test_golden_gpu_mixed(golden):
    import torch
    from paper_1709_04794_gb300 import sda
    p, g = golden
    op = sda.Operator(p, compute="f16")
    ns = len(p.shifts)
    w = torch.empty((1, ns, p.d), dtype=torch.float64, device="cuda")
    o = sda.sda_default_opts()
    tol = 1e-6
    o.tol, o.max_iter = tol, 20000
    code, rep = sda.sda_solve_shifts(op.handle, p.shifts, o, w_out=w, n_report=1)
    assert code == sda.SDA_OK
    ob = oracle.from_problem(p)
    b = ob.rhs_canonical()
    W = w[0].cpu().numpy()
    for s, beta in enumerate(p.shifts):
        assert ob.true_residual(b, beta, W[s]) < 20 * tol, s


MODES = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "small_300x96_modes_fp64.json")


@pytest.fixture(scope="module")
def modes():
    return json.load(open(MODES))


def test_golden_regression_mode(golden, modes):
    """CSR-SDA's regression step (Algorithm 5, line 5) on the stored X: the
    oracle reproduces the stored solutions, which solve (X^T X + beta I) w = X^T z."""
    p, g = golden
    m = modes["regression"]
    X = oracle.dense_x(p.x_ptr, p.x_col, p.x_val, p.d)
    b = np.asarray(m["rhs"])
    assert np.allclose(b, X.T @ np.asarray(m["z"]), rtol=1e-13, atol=1e-12)
    o = oracle.Oracle.regression(p.x_ptr, p.x_col, p.x_val, p.d)
    res = o.shifted_cg(b, p.shifts, tol=1e-13, max_iter=50000)
    assert res.iters.tolist() == m["iters"]
    for s, beta in enumerate(p.shifts):
        w = np.asarray(m["w"][s])
        assert _rel(res.W[s], w) < 1e-12, s
        assert _rel(w, np.linalg.solve(X.T @ X + beta * np.eye(p.d), b)) < 1e-9, s


def test_golden_sa_mode(golden, modes):
    """SA-SDA (Algorithm 6) on the stored graph and labels: the oracle with
    X = I_N reproduces the stored ratings, which solve (M - omega 1_l 1_l^T / l
    + beta I) z = d."""
    p, g = golden
    m = modes["sa"]
    n, y, a = p.n, p.labels[0], p.alpha
    o = oracle.Oracle(np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n),
                      p.s_ptr, p.s_col, p.s_val, y, n, a)
    d = o.rhs_canonical()
    assert np.array_equal(d, np.asarray(m["rhs"]))
    res = o.shifted_cg(d, p.shifts, tol=1e-13, max_iter=50000)
    assert res.iters.tolist() == m["iters"]
    Sd = np.zeros((n, n))
    for i in range(n):
        Sd[i, p.s_col[p.s_ptr[i]:p.s_ptr[i + 1]]] = p.s_val[p.s_ptr[i]:p.s_ptr[i + 1]]
    one_l = (y != 0).astype(float)
    om = 1.0 - a
    Mt = om * np.diag(one_l) + a * (np.diag(Sd.sum(1)) - Sd) - om * np.outer(one_l, one_l) / one_l.sum()
    for s, beta in enumerate(p.shifts):
        z = np.asarray(m["z"][s])
        assert _rel(res.W[s], z) < 1e-12, s
        assert _rel(z, np.linalg.solve(Mt + beta * np.eye(n), d)) < 1e-9, s
