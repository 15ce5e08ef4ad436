"""The differentiable hyperparameter fit at its workload's size: 500,000 x
262,144 binary X stored in FP8 (e4m3), 50 nonzeros per row, 64 targets,
held-out logistic loss, gradient in (alpha, beta) by the batched adjoint
(sda_adjoint_grad_batched) behind a torch.autograd.Function.

* Subsample (5,000 rows: the labelled and held-out rows of the four targets
  with the smallest labelled sets, filled with seeded random rows; the graph
  restricted to those rows): the batched adjoint gradients of the FP64 path
  and of the FP8 path refined to FP64 residuals equal the FP64 oracle's
  (C oracle CG, sparse products; pinned against the dense gradient on the
  CPU) within 1e-6 relative.
* Full size: the gradient of the mean held-out loss of all 64 targets at a
  common (alpha, beta), FP8 path refined to an FP64 residual of 1e-10, equals
  central finite differences (h = 1e-4 on alpha and on log beta) of the same
  loss within 1e-3 relative (the loss itself is accurate to ~1e-10, so the
  differences carry ~1e-6 of noise relative to the loss).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_04794_gb300 import autograd, sda, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg4():
    return synth.make_problem("adjoint_64t_500k")


def _subsample(p, n_keep=5000, n_tg=4, seed=17):
    ell = (p.labels != 0).sum(axis=1)
    tg = np.argsort(ell, kind="stable")[:n_tg]
    keep = set()
    for t in tg:
        keep.update(np.nonzero(p.labels[t])[0].tolist())
        keep.update(p.heldout[t].tolist())
    rng = np.random.default_rng(seed)
    while len(keep) < n_keep:
        keep.update(rng.integers(0, p.n, n_keep - len(keep)).tolist())
    rows = np.array(sorted(keep), dtype=np.int64)
    new_id = -np.ones(p.n, dtype=np.int64)
    new_id[rows] = np.arange(rows.size)
    cnt = np.diff(p.x_ptr)[rows]
    x_ptr = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    sel = np.concatenate([np.arange(p.x_ptr[i], p.x_ptr[i + 1]) for i in rows])
    x_col, x_val = p.x_col[sel], p.x_val[sel]
    s_rows, s_cols, s_vals = [], [], []
    for k, i in enumerate(rows):
        c = p.s_col[p.s_ptr[i]:p.s_ptr[i + 1]]
        v = p.s_val[p.s_ptr[i]:p.s_ptr[i + 1]]
        m = new_id[c] >= 0
        s_cols.append(new_id[c[m]])
        s_vals.append(v[m])
        s_rows.append(np.full(int(m.sum()), k))
    s_cnt = np.bincount(np.concatenate(s_rows), minlength=rows.size)
    s_ptr = np.concatenate([[0], np.cumsum(s_cnt)]).astype(np.int64)
    labels = p.labels[tg][:, rows]
    truth = p.truth[tg][:, rows]
    held = [new_id[p.heldout[t]] for t in tg]
    return synth.Problem(p.workload, x_ptr, x_col.astype(np.int32), x_val, s_ptr,
                         np.concatenate(s_cols).astype(np.int32), np.concatenate(s_vals), labels, truth, held,
                         p.shifts, p.alpha)


def _adjoint(op, sub, alpha, beta, compute, refine):
    T, d = sub.labels.shape[0], sub.d
    o = sda.sda_default_opts()
    o.tol, o.max_iter, o.batch_targets, o.alpha = 1e-12, 50000, 1, alpha
    if refine:
        o.tol, o.refine_rounds, o.refine_tol = 1e-4, 12, 1e-12
    w = torch.empty((T, 1, d), dtype=torch.float64, device="cuda")
    sda.sda_solve_shifts(op.handle, [beta], o, w_out=w, n_report=T)
    rows = np.concatenate(sub.heldout)
    off = np.concatenate([[0], np.cumsum([h.size for h in sub.heldout])])
    g = np.empty(rows.size)
    for t in range(T):
        r = sub.heldout[t]
        sc = torch.empty((1, r.size), dtype=torch.float64, device="cuda")
        sda.sda_project_rows(op.handle, w[t, 0], 1, torch.from_numpy(r).cuda(), sc, 1, t)
        _, g[off[t]:off[t + 1]] = oracle.logistic_loss(sc[0].cpu().numpy(), sub.truth[t][r])
    oa = sda.sda_default_opts()
    oa.tol, oa.max_iter = o.tol, 50000
    oa.refine_rounds, oa.refine_tol = o.refine_rounds, o.refine_tol
    code, da, db, rep = sda.sda_adjoint_grad_batched(op.handle, list(range(T)), alpha, [beta] * T,
                                                     w[:, 0].contiguous(), torch.from_numpy(g).cuda(),
                                                     torch.from_numpy(rows).cuda(), off, oa)
    assert code == sda.SDA_OK, rep
    return da, db


@pytest.mark.parametrize("compute,refine", [("f64", False), ("f8e4m3", True)])
def test_config4_subsample_adjoint_matches_oracle(cfg4, compute, refine):
    sub = _subsample(cfg4)
    alpha = 0.1
    op = sda.Operator(sub, compute=compute, alpha=alpha)
    for beta in (1e-2, 1.0):
        da, db = _adjoint(op, sub, alpha, beta, compute, refine)
        for t in range(sub.labels.shape[0]):
            o = oracle.from_problem(sub, target=t, alpha=alpha)
            _, ra, rb, _ = oracle.adjoint_grad_sparse(o, sub.x_ptr, sub.x_col, sub.x_val, sub.s_ptr, sub.s_col,
                                                      sub.s_val, sub.heldout[t], sub.truth[t][sub.heldout[t]],
                                                      beta, tol=1e-13)
            assert abs(da[t] - ra) <= 1e-6 * abs(ra) + 1e-14, (beta, t, da[t], ra)
            assert abs(db[t] - rb) <= 1e-6 * abs(rb) + 1e-14, (beta, t, db[t], rb)


def test_config4_full_size_gradient_matches_finite_differences(cfg4):
    op = sda.Operator(cfg4, compute="f8e4m3")
    T = cfg4.labels.shape[0]
    rows = torch.from_numpy(np.concatenate(cfg4.heldout)).cuda()
    off = np.concatenate([[0], np.cumsum([h.size for h in cfg4.heldout])])
    yr = torch.from_numpy(np.concatenate([cfg4.truth[t][cfg4.heldout[t]] for t in range(T)]).astype(np.float64)).cuda()
    kw = dict(tol=1e-4, max_iter=50000, refine_rounds=12, refine_tol=1e-10)
    alpha, beta = 0.1, 1.0

    def f(al, be):
        return autograd.held_out_loss_batched(torch.tensor(al, dtype=torch.float64),
                                              torch.tensor(be, dtype=torch.float64), op, 0, T, rows, off, yr,
                                              **kw).item()

    a = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    b = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
    autograd.held_out_loss_batched(a, b, op, 0, T, rows, off, yr, **kw).backward()
    h = 1e-4
    fd_a = (f(alpha + h, beta) - f(alpha - h, beta)) / (2 * h)
    fd_lb = (f(alpha, beta * np.exp(h)) - f(alpha, beta * np.exp(-h))) / (2 * h)
    assert abs(a.grad.item() - fd_a) <= 1e-3 * abs(fd_a), (a.grad.item(), fd_a)
    assert abs(beta * b.grad.item() - fd_lb) <= 1e-3 * abs(fd_lb), (beta * b.grad.item(), fd_lb)
