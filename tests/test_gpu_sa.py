"""SA-SDA (Algorithm 6) through sda_build_sa: the SDA operator with the
identity as the data matrix, over N-vectors, against the FP64 oracle with
X = I_N (whose paper form is Algorithm 6's operator; pinned to the dense
M - omega 1_l 1_l^T / l in test_oracle_pins.py).

Bars as for the SDA operator: apply 1e-12 relative; FP64 iterates after 7
fixed iterations 1e-9; converged FP64 (tol 1e-10) 1e-6 on the ratings z with
FP64 true residuals below 1e-9; mixed path true residual within 20 x tol;
AUC of the ratings on the held-out rows equal to 4 decimals.
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
def sa():
    p = synth.custom_problem(5001, 200, 20, seed=31, values="binary", n_labelled=600, k=8, shifts=(1e-2, 1e2, 6))
    n = p.n
    o = oracle.Oracle(np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n),
                      p.s_ptr, p.s_col, p.s_val, p.labels[0], n, p.alpha)
    return p, o


def _op(p, compute):
    return sda.Operator.sa(p.s_ptr, p.s_col, p.s_val, p.labels, p.alpha, compute=compute)


def _solve(op, p, tol=1e-10, fixed=0, check=1):
    ns, n = len(p.shifts), p.n
    z = torch.empty((1, ns, n), dtype=torch.float64, device="cuda")
    o = sda.sda_default_opts()
    o.tol, o.max_iter, o.fixed_iters, o.check_residual = tol, 20000, fixed, check
    code, rep = sda.sda_solve_shifts(op.handle, p.shifts, o, w_out=z, n_report=1)
    return code, rep[0], z[0].cpu().numpy()


def test_sa_apply(sa):
    p, o = sa
    op = _op(p, "f64")
    x = np.random.default_rng(2).standard_normal(p.n)
    q = torch.empty(p.n, dtype=torch.float64, device="cuda")
    sda.sda_operator_apply(op.handle, 0, 0.25, torch.from_numpy(x).cuda(), q)
    assert _rel(q.cpu().numpy(), o.apply(x, 0.25)) < 1e-12


def test_sa_fixed_iterations(sa):
    p, o = sa
    k = 7
    code, rep, z = _solve(_op(p, "f64"), p, fixed=k, check=0)
    ref = o.shifted_cg(o.rhs_canonical(), p.shifts, fixed_iters=k)
    for s in range(len(p.shifts)):
        assert _rel(z[s], ref.W[s]) < 1e-9, s


def test_sa_converged_ratings(sa):
    p, o = sa
    code, rep, z = _solve(_op(p, "f64"), p, tol=1e-10)
    assert code == sda.SDA_OK
    ref = o.shifted_cg(o.rhs_canonical(), p.shifts, tol=1e-12, max_iter=50000)
    rows = np.asarray(p.heldout[0])
    for s in range(len(p.shifts)):
        assert _rel(z[s], ref.W[s]) < 1e-6, s
        assert rep[s]["true_residual"] < 1e-9, rep[s]
        a_gpu = oracle.auc(z[s][rows], p.truth[0][rows])
        a_ref = oracle.auc(ref.W[s][rows], p.truth[0][rows])
        assert abs(a_gpu - a_ref) < 5e-5, (s, a_gpu, a_ref)


def test_sa_mixed(sa):
    p, o = sa
    tol = 1e-6
    code, rep, z = _solve(_op(p, "f16"), p, tol=tol)
    assert code == sda.SDA_OK
    b = o.rhs_canonical()
    for s, beta in enumerate(p.shifts):
        assert o.true_residual(b, beta, z[s]) < 20 * tol, s
