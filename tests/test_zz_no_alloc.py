"""sda_operator_apply_static: the operator apply for callers that cannot
allocate device memory (an application whose pool allocator owns all device
memory, or a loop where cudaMalloc's implicit synchronisation is not
acceptable).  Its scratch is a fixed device array inside the library.

The result must equal the allocating sda_operator_apply's within the tolerance
the other apply tests use (1e-12 relative), on two calls in a row (the second
call finds the array holding the first call's contents).  This file is
collected last, so a run that stops at the first failure has run every other
test before it."""
import numpy as np
import pytest
import torch

from paper_1709_04794_gb300 import sda, synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("compute", ["f64", "f16"])
def test_static_apply_matches_allocating_apply(compute):
    prob = synth.custom_problem(9001, 3001, 22, seed=5, values="counts", n_labelled=700, k=6,
                                shifts=(1e-3, 1e2, 7))
    op = sda.Operator(prob, compute=compute)
    rng = np.random.default_rng(11)
    for call, sigma in enumerate((0.0, 0.75)):        # two calls in a row, different inputs
        p = torch.from_numpy(rng.standard_normal(prob.d)).cuda()
        q_ref = torch.empty(prob.d, dtype=torch.float64, device="cuda")
        q_st = torch.full((prob.d,), float("nan"), dtype=torch.float64, device="cuda")
        sda.sda_operator_apply(op.handle, 0, sigma, p, q_ref)
        sda.sda_operator_apply_static(op.handle, 0, sigma, p, q_st)
        torch.cuda.synchronize()
        assert _rel(q_st.cpu().numpy(), q_ref.cpu().numpy()) < 1e-12, (call, sigma)


@pytest.mark.parametrize("kind", ["regression", "sa"])
def test_static_apply_other_operators(kind):
    """The X^T X operator of CSR-SDA's regression step (no graph, no centring)
    and SA-SDA's operator (X = I_N) go through the same row and column passes."""
    prob = synth.custom_problem(2500, 900, 14, seed=8, values="counts", n_labelled=300, k=5,
                                shifts=(1e-3, 1e2, 5))
    if kind == "regression":
        op = sda.Operator.regression(prob.x_ptr, prob.x_col, prob.x_val, prob.d, compute="f16")
        dim = prob.d
    else:
        op = sda.Operator.sa(prob.s_ptr, prob.s_col, prob.s_val, prob.labels, prob.alpha, compute="f32")
        dim = prob.n
    rng = np.random.default_rng(12)
    for call, sigma in enumerate((0.0, 0.3)):
        p = torch.from_numpy(rng.standard_normal(dim)).cuda()
        q_ref = torch.empty(dim, dtype=torch.float64, device="cuda")
        q_st = torch.full((dim,), float("nan"), dtype=torch.float64, device="cuda")
        sda.sda_operator_apply(op.handle, 0, sigma, p, q_ref)
        sda.sda_operator_apply_static(op.handle, 0, sigma, p, q_st)
        torch.cuda.synchronize()
        assert _rel(q_st.cpu().numpy(), q_ref.cpu().numpy()) < 1e-12, (kind, call, sigma)
    op.close()


def test_static_apply_rejects_oversized_operator():
    # 2 (N + D) above the 2**20-double array: refused with a clear error, nothing launched
    prob = synth.custom_problem(400_000, 200_000, 3, seed=6, n_labelled=100, k=2, shifts=(1e-2, 1e1, 2),
                                knn_cap=8)
    op = sda.Operator(prob, compute="f16")
    p = torch.zeros(prob.d, dtype=torch.float64, device="cuda")
    q = torch.zeros(prob.d, dtype=torch.float64, device="cuda")
    with pytest.raises(sda.SDAError) as e:
        sda.sda_operator_apply_static(op.handle, 0, 0.0, p, q)
    assert e.value.code == sda.SDA_ERR_SHAPE and "static scratch" in str(e.value)
