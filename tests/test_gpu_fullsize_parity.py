"""Full-size parity of the mixed path with per-shift FP64 refinement against
the FP64 oracle, at the converged-solution parity bar (parity.py): 1e-6 relative on w,
norm-wise and element-wise, on every shift whose residual bound
kappa_s (rho + rho*) permits it, else the error reported beside that bound;
AUC of the held-out rows equal to 4 decimals.

Workloads: the single-target 200,000 x 131,072 FP16 problem (32 shifts
1e-5..1e3) and the first target of the first batch of the 256-target problem
(batched path, 16 shifts).  The GPU solves to tol 1e-3 (the paper's Table 6
tolerance) and refines every (target, shift) to an FP64 true residual of
1e-11.  The oracle runs shifted CG (Algorithm 3) to tol 1e-12 with an
iteration cap of 6,000: the shifts above about 0.1 converge within it; on the
smallest shifts (kappa up to ~1e8, 17,691 iterations to 1e-12) it stops at
the cap and its own FP64 true residual enters the bound, so those errors are
reported, not asserted at 1e-6.  The GPU's FP64 true residuals are checked
with the oracle's own operator on every shift.
"""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_1709_04794_gb300 import sda, synth

pytestmark = pytest.mark.gpu

RTOL = 1e-11
ORACLE_CAP = 6000


def _against_oracle(prob, t, wg, reps, shifts):
    ob = oracle.from_problem(prob, target=t)
    b = ob.rhs_canonical()
    ref = ob.shifted_cg(b, shifts, tol=1e-12, max_iter=ORACLE_CAP)
    lam = parity.lambda_max(ob, iters=40)
    rows = prob.heldout[t]
    truth = prob.truth[t][rows]
    asserted = 0
    for s, beta in enumerate(shifts):
        rho = ob.true_residual(b, beta, wg[s])
        assert reps[s]["status"] == sda.SDA_OK and reps[s]["true_residual"] <= RTOL, (s, reps[s])
        assert rho <= 2 * RTOL, (s, rho)
        res = parity.compare(wg[s], ref.W[s], beta, lam, rho, ob.true_residual(b, beta, ref.W[s]))
        parity.check(res, (t, s))
        asserted += res["asserted"]
        a_gpu = oracle.auc(ob.project(wg[s])[rows], truth)
        a_ref = oracle.auc(ob.project(ref.W[s])[rows], truth)
        if res["asserted"]:
            assert abs(a_gpu - a_ref) < parity.AUC_BAR, (s, a_gpu, a_ref)
        else:
            print("AUC beside the oracle's capped run:", (t, s), a_gpu, a_ref)
    # the larger half of the shifts reach the 1e-6 bar
    assert asserted >= len(shifts) // 3, asserted


def test_single_target_200k_refined_matches_oracle():
    p = synth.make_problem("single_mixed_200k")
    op = sda.Operator(p, compute="f16")
    ns = len(p.shifts)
    w = torch.empty((1, ns, p.d), dtype=torch.float64, device="cuda")
    o = sda.sda_default_opts()
    o.tol, o.max_iter, o.refine_rounds, o.refine_tol = 1e-3, 20000, 12, RTOL
    code, rep = sda.sda_solve_shifts(op.handle, p.shifts, o, w_out=w, n_report=1)
    assert code == sda.SDA_OK
    op.close()
    _against_oracle(p, 0, w[0].cpu().numpy(), rep[0], p.shifts)


def test_batched_200k_first_batch_refined_matches_oracle():
    p = synth.make_problem("batched_256t_200k", n_targets=16)
    op = sda.Operator(p, compute="f16")
    nt, ns = 16, len(p.shifts)
    w = torch.empty((nt, ns, p.d), dtype=torch.float64, device="cuda")
    o = sda.sda_default_opts()
    o.tol, o.max_iter, o.batch_targets = 1e-3, 20000, 1
    o.refine_rounds, o.refine_tol = 12, RTOL
    code, rep = sda.sda_solve_shifts(op.handle, p.shifts, o, w_out=w, n_report=nt)
    assert code == sda.SDA_OK
    for t in range(nt):
        for r in rep[t]:
            assert r["status"] == sda.SDA_OK and r["true_residual"] <= RTOL, (t, r)
    op.close()
    _against_oracle(p, 0, w[0].cpu().numpy(), rep[0], p.shifts)
