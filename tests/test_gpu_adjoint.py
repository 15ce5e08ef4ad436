"""Adjoint gradient of the held-out loss (A12): against the oracle's dense
gradient and against central finite differences (h = 1e-4 on alpha and on
log beta) of the GPU loss itself."""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_04794_gb300 import autograd, sda, synth

pytestmark = pytest.mark.gpu


def _setup(prob, compute):
    op = sda.Operator(prob, compute=compute)
    rows = torch.from_numpy(prob.heldout[0]).cuda()
    yr = torch.from_numpy(prob.truth[0][prob.heldout[0]].astype(np.float64)).cuda()
    return op, rows, yr


def test_adjoint_matches_dense_oracle(tiny):
    op, rows, yr = _setup(tiny, "f64")
    alpha, beta = 0.3, 0.05
    a = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    b = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
    loss = autograd.held_out_loss(a, b, op, 0, rows, yr, tol=1e-13)
    loss.backward()
    X = oracle.dense_x(tiny.x_ptr, tiny.x_col, tiny.x_val, tiny.d)
    ref_loss, ref_da, ref_db, _ = oracle.adjoint_grad_dense(X, tiny.s_ptr, tiny.s_col, tiny.s_val, tiny.labels[0],
                                                            alpha, beta, tiny.heldout[0],
                                                            tiny.truth[0][tiny.heldout[0]])
    assert abs(loss.item() - ref_loss) <= 1e-9 * abs(ref_loss)
    assert abs(a.grad.item() - ref_da) <= 1e-6 * abs(ref_da) + 1e-12
    assert abs(b.grad.item() - ref_db) <= 1e-6 * abs(ref_db) + 1e-12


def test_adjoint_matches_finite_differences(cfg1):
    """FP64 path: the adjoint gradient against central differences of the loss."""
    compute, rtol, tol = "f64", 1e-4, 1e-12
    op, rows, yr = _setup(cfg1, compute)
    alpha, beta = 0.1, 0.05

    def f(al, be):
        return autograd.held_out_loss(torch.tensor(al, dtype=torch.float64),
                                      torch.tensor(be, dtype=torch.float64), op, 0, rows, yr, tol=tol).item()

    a = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    b = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
    autograd.held_out_loss(a, b, op, 0, rows, yr, tol=tol).backward()
    h = 1e-4
    fd_a = (f(alpha + h, beta) - f(alpha - h, beta)) / (2 * h)
    fd_lb = (f(alpha, beta * np.exp(h)) - f(alpha, beta * np.exp(-h))) / (2 * h)
    assert abs(a.grad.item() - fd_a) <= rtol * abs(fd_a) + 1e-10, (a.grad.item(), fd_a)
    assert abs(beta * b.grad.item() - fd_lb) <= rtol * abs(fd_lb) + 1e-10, (beta * b.grad.item(), fd_lb)


def test_mixed_adjoint_close_to_fp64_adjoint(cfg1):
    """Mixed path (FP16 X, FP32 vectors): finite differences of its loss are below
    the solve's noise at this gradient size, so it is compared with the FP64
    adjoint instead; both solves to 1e-8, agreement to 5 %."""
    grads = {}
    for compute in ("f64", "f16"):
        op, rows, yr = _setup(cfg1, compute)
        a = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
        b = torch.tensor(0.05, dtype=torch.float64, requires_grad=True)
        autograd.held_out_loss(a, b, op, 0, rows, yr, tol=1e-8).backward()
        grads[compute] = (a.grad.item(), b.grad.item())
    for k in range(2):
        assert abs(grads["f16"][k] - grads["f64"][k]) <= 5e-2 * abs(grads["f64"][k]), grads


def test_adjoint_rejects_bad_rows(tiny):
    op, rows, yr = _setup(tiny, "f64")
    w = torch.zeros(tiny.d, dtype=torch.float64, device="cuda")
    bad = torch.tensor([0, tiny.n], dtype=torch.int64, device="cuda")
    g = torch.ones(2, dtype=torch.float64, device="cuda")
    with pytest.raises(sda.SDAError) as e:
        sda.sda_adjoint_grad(op.handle, 0, float("nan"), 0.1, w, g, bad)
    assert e.value.code == sda.SDA_ERR_INVALID_ARG


def test_alpha_override_matches_rebuilt_operator(cfg1):
    """Solving with opts.alpha equals building the operator with that alpha."""
    op1 = sda.Operator(cfg1, compute="f64", alpha=0.1)
    op2 = sda.Operator(cfg1, compute="f64", alpha=0.4)
    ns = len(cfg1.shifts)
    w1 = torch.empty((1, ns, cfg1.d), dtype=torch.float64, device="cuda")
    w2 = torch.empty_like(w1)
    o = sda.sda_default_opts()
    o.fixed_iters = 15
    o.alpha = 0.4
    sda.sda_solve_shifts(op1.handle, cfg1.shifts, o, w_out=w1, n_report=1)
    o2 = sda.sda_default_opts()
    o2.fixed_iters = 15
    sda.sda_solve_shifts(op2.handle, cfg1.shifts, o2, w_out=w2, n_report=1)
    assert torch.equal(w1, w2)
