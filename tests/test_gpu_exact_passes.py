"""The X passes of the FP64 residual check (and of the other FP64 block
utilities: projections, adjoint contractions, class sums) run in exact fixed
point when every value of X is a small integer times one power of two (binary
and count data), else in FP64 arithmetic.  Both are checked against the
oracle's FP64 true residual ||b - (B + beta I) w|| / ||b|| of the same GPU
solutions.  Six fixed iterations leave residuals of 1e-1 .. 1e-4, far above
the rounding floor of either evaluation, so the reported residuals must equal
the oracle's to 1e-9 relative.  The operator info says which arithmetic ran.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_1709_04794_gb300 import sda, synth

pytestmark = pytest.mark.gpu


def _problem(values):
    p = synth.custom_problem(1800, 900, 16, seed=51, values="counts" if values in ("counts", "signed") else "binary",
                             n_targets=2, n_labelled=150, k=5, shifts=(1e-3, 1e1, 5))
    if values == "real":
        # values spread over many binary digits (exact in FP32): no common power-of-two grid
        x = np.random.default_rng(52).uniform(0.1, 2.0, p.x_val.size).astype(np.float32).astype(np.float64)
        p = dataclasses.replace(p, x_val=x)
    if values == "signed":
        # counts with random signs: x_int = x, |x_int| < 2^4, negative products
        sign = np.where(np.random.default_rng(55).random(p.x_val.size) < 0.5, -1.0, 1.0)
        p = dataclasses.replace(p, x_val=p.x_val * sign)
    if values == "quarters":
        # multiples of 1/4 up to 7.75: x_int = 4 x < 2^5, two fraction bits
        x = np.random.default_rng(53).integers(1, 32, p.x_val.size) / 4.0
        p = dataclasses.replace(p, x_val=x)
    return p


@pytest.mark.parametrize("batch", [0, 1])
@pytest.mark.parametrize("values,compute,expect,bits", [
    ("binary", "f8e4m3", 1, (0, 1)),
    ("binary", "f64", 1, (0, 1)),
    ("binary", "pattern", 1, (0, 1)),
    ("counts", "f16", 1, (0, 4)),
    ("signed", "f16", 1, (0, 4)),
    ("quarters", "f16", 1, (2, 5)),
    ("real", "f32", -1, None),
    ("real", "f64", -1, None),
])
def test_residual_check_matches_oracle(values, compute, expect, bits, batch):
    p = _problem(values)
    op = sda.Operator(p, compute=compute)
    T, ns, d = 2, len(p.shifts), p.d
    o = sda.sda_default_opts()
    o.fixed_iters, o.batch_targets, o.check_residual = 6, batch, 1
    w = torch.empty((T, ns, d), dtype=torch.float64, device="cuda")
    code, rep = sda.sda_solve_shifts(op.handle, p.shifts, o, w_out=w, n_report=T)
    assert code == sda.SDA_OK
    info = sda.sda_get_operator_info(op.handle)
    assert info["exact_x_passes"] == expect, info
    if bits is not None:
        assert (info["x_frac_bits"], info["x_int_bits"]) == bits, info
    wh = w.cpu().numpy()
    for t in range(T):
        ob = oracle.from_problem(p, target=t)
        b = ob.rhs_canonical()
        for s, beta in enumerate(p.shifts):
            ref = ob.true_residual(b, beta, wh[t, s])
            got = rep[t][s]["true_residual"]
            assert 1e-5 < ref < 1.0, (t, s, ref)
            assert abs(got - ref) <= 1e-9 * ref, (values, compute, t, s, got, ref)


def test_projection_exact_passes_match_oracle():
    """Projections of FP64 vectors spanning six decades through the fixed-point
    row pass: X w and the centred X w - <mu, w> equal the oracle's element-wise
    to 1e-13 of the largest entry."""
    p = _problem("counts")
    op = sda.Operator(p, compute="f16")
    rng = np.random.default_rng(54)
    W = rng.standard_normal((3, p.d)) * np.logspace(-3, 3, p.d)[None, :]
    sc = torch.empty((3, p.n), dtype=torch.float64, device="cuda")
    ob = oracle.from_problem(p, target=0)
    mu, _, _, _ = ob.class_means()
    for centred in (0, 1):
        sda.sda_project(op.handle, torch.from_numpy(W).cuda(), 3, sc, centred, 0)
        assert sda.sda_get_operator_info(op.handle)["exact_x_passes"] == 1
        for v in range(3):
            ref = ob.project(W[v]) - (mu @ W[v] if centred else 0.0)
            got = sc[v].cpu().numpy()
            assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref)), (centred, v)
