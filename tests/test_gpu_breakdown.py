"""Failure detection on the host side: inputs that would poison the Krylov
run are injected on the host and must come back as error codes, with the
operator still usable afterwards (nothing here faults or hangs the GPU).

* a right-hand side holding a NaN or an infinity (rhs_mode SDA_RHS_GIVEN)
  stops the shifted CG before its first iteration with SDA_ERR_BREAKDOWN
  (single target and batched targets, FP64 and mixed paths);
* a non-finite value of X is refused by the build (SDA_ERR_VALUE_NOT_EXACT),
  a non-finite weight of S likewise (SDA_ERR_NOT_SYMMETRIC);
* after a breakdown the same operator solves a valid system normally
  (refined to an FP64 true residual of 1e-8);
* the opposite case: a residual that vanishes exactly in a fixed-iteration run
  (underflow at a shift far above ||B||) is an exact solution, not a breakdown.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_04794_gb300 import sda, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def prob():
    return synth.custom_problem(1500, 700, 18, seed=41, values="counts", n_targets=3, n_labelled=200, k=5,
                                shifts=(1e-3, 1e1, 4))


def _opts(batch, tol=1e-8):
    o = sda.sda_default_opts()
    o.tol, o.max_iter, o.rhs_mode, o.batch_targets = tol, 5000, sda.SDA_RHS_GIVEN, batch
    return o


@pytest.mark.parametrize("compute", ["f64", "f16"])
@pytest.mark.parametrize("batch", [0, 1])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_rhs_is_a_breakdown(prob, compute, batch, bad):
    op = sda.Operator(prob, compute=compute)
    T, ns, d = 3, len(prob.shifts), prob.d
    rhs = np.random.default_rng(2).standard_normal((T, d))
    rhs[1, d // 3] = bad
    w = torch.empty((T, ns, d), dtype=torch.float64, device="cuda")
    with pytest.raises(sda.SDAError) as e:
        sda.sda_solve_shifts(op.handle, prob.shifts, _opts(batch), w_out=w, n_report=T,
                             rhs=torch.from_numpy(rhs).cuda())
    assert e.value.code == sda.SDA_ERR_BREAKDOWN, str(e.value)
    # the operator (and the CUDA context) stay usable: the same systems with a
    # finite right-hand side, refined to an FP64 true residual of 1e-8 (a random
    # right-hand side leaves the FP32 vectors of the mixed path near 1e-4 unrefined)
    rhs[1, d // 3] = 0.5
    o = _opts(batch, tol=1e-6)
    o.refine_rounds, o.refine_tol = 6, 1e-8
    code, rep = sda.sda_solve_shifts(op.handle, prob.shifts, o, w_out=w, n_report=T,
                                     rhs=torch.from_numpy(rhs).cuda())
    assert code == sda.SDA_OK
    for t in range(T):
        for r in rep[t]:
            assert r["status"] == sda.SDA_OK and r["true_residual"] <= 1e-8, (t, r)


def test_nonfinite_x_value_refused_by_build(prob):
    x_val = prob.x_val.copy()
    x_val[17] = float("nan")
    with pytest.raises(sda.SDAError) as e:
        sda.sda_build_operator(prob.x_ptr, prob.x_col, x_val, prob.d, prob.s_ptr, prob.s_col, prob.s_val,
                               prob.labels, prob.alpha, float("nan"), "f64")
    assert e.value.code == sda.SDA_ERR_VALUE_NOT_EXACT


def test_nonfinite_graph_weight_refused_by_build(prob):
    s_val = prob.s_val.copy()
    s_val[5] = float("inf")
    with pytest.raises(sda.SDAError) as e:
        sda.sda_build_operator(prob.x_ptr, prob.x_col, prob.x_val, prob.d, prob.s_ptr, prob.s_col, s_val,
                               prob.labels, prob.alpha, float("nan"), "f64")
    assert e.value.code == sda.SDA_ERR_NOT_SYMMETRIC


@pytest.mark.parametrize("compute", ["f64", "f16"])
@pytest.mark.parametrize("batch", [0, 1])
def test_exactly_vanished_residual_ends_a_fixed_run(compute, batch):
    """A fixed-iteration run at a shift far above ||B|| converges until its
    residual underflows to exactly zero (within ~20 iterations in FP32 vectors,
    ~150 in FP64). That is an exact solution, not a breakdown: the run ends
    there with SDA_OK, and the solution equals the oracle's to the vectors'
    precision."""
    p = synth.custom_problem(1200, 500, 12, seed=43, values="counts", n_targets=2, n_labelled=150, k=5,
                             shifts=(1e5, 1e5, 1))
    op = sda.Operator(p, compute=compute)
    w = torch.empty((2, 1, p.d), dtype=torch.float64, device="cuda")
    o = sda.sda_default_opts()
    o.fixed_iters, o.batch_targets, o.check_residual = 400, batch, 1
    code, rep = sda.sda_solve_shifts(op.handle, p.shifts, o, w_out=w, n_report=2)
    assert code == sda.SDA_OK
    wh = w.cpu().numpy()
    for t in range(2):
        assert rep[t][0]["status"] == sda.SDA_OK, rep[t]
        assert rep[t][0]["iters"] < 400, rep[t]
        ob = oracle.from_problem(p, target=t)
        ref = ob.shifted_cg(ob.rhs_canonical(), p.shifts, tol=1e-14).W[0]
        bar = 1e-12 if compute == "f64" else 1e-6
        assert np.linalg.norm(wh[t, 0] - ref) <= bar * np.linalg.norm(ref), (t, rep[t])
