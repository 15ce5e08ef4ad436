"""Per-shift refinement of the mixed path (no paper counterpart): a shift whose
FP64 true residual exceeds refine_tol gets corrections c solved from
(B + beta I) c = b - (B + beta I) w in the iteration's precision and added in
FP64.  Refined, the FP16/FP32 solve reaches FP64-level residuals; its solution
is then compared with the FP64 oracle's at the same residual.

Bar: every shift's FP64 true residual <= refine_tol (1e-11); w against the
FP64 oracle (tol 1e-13) within 1e-6 norm-wise and element-wise on every shift
whose residual bound kappa_s (rho + rho*) permits it, else within that bound
(reported); AUC equal to 4 decimals on every shift (parity.py).
"""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_1709_04794_gb300 import sda

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _solve(prob, compute, tol, rounds=0, rtol=float("nan"), max_iter=20000):
    op = sda.Operator(prob, compute=compute)
    ns, d = len(prob.shifts), prob.d
    w = torch.empty((1, ns, d), dtype=torch.float64, device="cuda")
    o = sda.sda_default_opts()
    o.tol, o.max_iter = tol, max_iter
    o.refine_rounds, o.refine_tol = rounds, rtol
    code, rep = sda.sda_solve_shifts(op.handle, prob.shifts, o, w_out=w, n_report=1)
    return code, rep[0], w[0].cpu().numpy()


def test_refined_mixed_reaches_fp64_residual(cfg1):
    rtol = 1e-11
    code, rep, w = _solve(cfg1, "f16", 1e-4, rounds=12, rtol=rtol)
    assert code == sda.SDA_OK
    for r in rep:
        assert r["status"] == sda.SDA_OK and r["true_residual"] <= rtol, r
    o = oracle.from_problem(cfg1)
    b = o.rhs_canonical()
    ref = o.shifted_cg(b, cfg1.shifts, tol=1e-13, max_iter=50000)
    lam = parity.lambda_max(o)
    rows = cfg1.heldout[0]
    y = cfg1.truth[0][rows]
    for s, beta in enumerate(cfg1.shifts):
        rho, rho_ref = o.true_residual(b, beta, w[s]), o.true_residual(b, beta, ref.W[s])
        assert rho <= 1.5 * rtol, (s, rho)
        parity.check(parity.compare(w[s], ref.W[s], beta, lam, rho, rho_ref), s)
        auc_gpu = oracle.auc(o.project(w[s])[rows], y)
        auc_ref = oracle.auc(o.project(ref.W[s])[rows], y)
        assert abs(auc_gpu - auc_ref) < parity.AUC_BAR, (s, auc_gpu, auc_ref)


def test_refinement_off_by_default(cfg1):
    code, rep, w = _solve(cfg1, "f16", 1e-4)
    code_r, rep_r, w_r = _solve(cfg1, "f16", 1e-4, rounds=0, rtol=1e-10)
    assert np.array_equal(w, w_r)
    assert [r["true_residual"] for r in rep] == [r["true_residual"] for r in rep_r]


def test_refinement_noop_when_already_below_target(cfg1):
    """A target above every shift's residual changes nothing."""
    code, rep, w = _solve(cfg1, "f16", 1e-6)
    code_r, rep_r, w_r = _solve(cfg1, "f16", 1e-6, rounds=3, rtol=1.0)
    assert np.array_equal(w, w_r)


def test_refinement_rejects_negative_rounds(cfg1):
    op = sda.Operator(cfg1, compute="f16")
    o = sda.sda_default_opts()
    o.refine_rounds = -1
    w = torch.empty((1, len(cfg1.shifts), cfg1.d), dtype=torch.float64, device="cuda")
    with pytest.raises(sda.SDAError) as e:
        sda.sda_solve_shifts(op.handle, cfg1.shifts, o, w_out=w, n_report=1)
    assert e.value.code == sda.SDA_ERR_INVALID_ARG
