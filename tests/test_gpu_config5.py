"""The largest workload at full size: 2,000,000 x 1,048,576 binary X stored in
FP8 (e4m3), 90M nonzeros, kNN graph k = 8 (26M nonzeros), 24 shifts; the first
16 of its 1,000 targets (one batch).  Outputs the FP64 oracle can compute one
by one at this size:

* the operator apply (B_t + sigma I) p of two targets: 1e-12 relative (the
  same bar as the small apply tests; X's values are exact in FP8);
* the batched FP64 path after 3 fixed iterations, two targets, every shift:
  1e-9 relative against the oracle's Algorithm 3 iterates;
* the FP64 true residual the mixed sweep reports after 70 iterations (the
  bench's protocol; fixed-point X passes) against the oracle's FP64 residual
  of the same solutions, two targets, every shift: 1e-9 relative, or 1e-13 of
  ||b|| where the residual nears the rounding floor of its own evaluation
  (b - (B + beta I) w cancels: at beta = 1e3, beta ||w|| is about ||b||, and two
  FP64 evaluations in different orders differ by ~1e-14 ||b||);
* the similarity graph built on the device: bit-exact against the input
  generator's (CSR pointers, columns, weights).
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_1709_04794_gb300 import sda, synth

pytestmark = pytest.mark.gpu

NT = 16
CHECK = (0, 5)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def cfg5():
    p = synth.make_problem("large_1000t_2m")
    return dataclasses.replace(p, labels=p.labels[:NT].copy(), truth=p.truth[:NT].copy(), heldout=p.heldout[:NT])


@pytest.fixture(scope="module")
def oracles(cfg5):
    return {t: oracle.from_problem(cfg5, target=t) for t in CHECK}


def test_config5_operator_apply_matches_oracle(cfg5, oracles):
    op = sda.Operator(cfg5, compute="f8e4m3")
    rng = np.random.default_rng(51)
    for t in CHECK:
        for sigma in (0.0, 0.3):
            p = rng.standard_normal(cfg5.d)
            q = torch.empty(cfg5.d, dtype=torch.float64, device="cuda")
            sda.sda_operator_apply(op.handle, t, sigma, torch.from_numpy(p).cuda(), q)
            assert _rel(q.cpu().numpy(), oracles[t].apply(p, sigma)) < 1e-12, (t, sigma)


def _sweep(prob, compute, fixed, check):
    op = sda.Operator(prob, compute=compute)
    ns = len(prob.shifts)
    w = torch.empty((NT, ns, prob.d), dtype=torch.float64, device="cuda")
    o = sda.sda_default_opts()
    o.fixed_iters, o.batch_targets, o.check_residual = fixed, 1, check
    code, rep = sda.sda_solve_shifts(op.handle, prob.shifts, o, w_out=w, n_report=NT)
    assert code == sda.SDA_OK
    return rep, w.cpu().numpy()


def test_config5_fp64_fixed_iterations_match_oracle(cfg5, oracles):
    k = 3
    _, w = _sweep(cfg5, "f64", k, 0)
    for t in CHECK:
        o = oracles[t]
        ref = o.shifted_cg(o.rhs_canonical(), cfg5.shifts, fixed_iters=k)
        for s in range(len(cfg5.shifts)):
            assert _rel(w[t, s], ref.W[s]) < 1e-9, (t, s, _rel(w[t, s], ref.W[s]))


def test_config5_mixed_sweep_residuals_match_oracle(cfg5, oracles):
    rep, w = _sweep(cfg5, "f8e4m3", 70, 1)
    for t in CHECK:
        o = oracles[t]
        b = o.rhs_canonical()
        for s, beta in enumerate(cfg5.shifts):
            ref = o.true_residual(b, beta, w[t, s])
            got = rep[t][s]["true_residual"]
            assert abs(got - ref) <= 1e-9 * ref + 1e-13, (t, s, got, ref)


def test_config5_knn_graph_matches_generator(cfg5):
    rp, col, val = sda.sda_knn_graph(torch.from_numpy(cfg5.x_ptr).cuda(), torch.from_numpy(cfg5.x_col).cuda(),
                                     cfg5.d, 8, 96)
    assert np.array_equal(rp.cpu().numpy(), cfg5.s_ptr)
    assert np.array_equal(col.cpu().numpy(), cfg5.s_col)
    assert np.array_equal(val.cpu().numpy(), cfg5.s_val)
