"""torch.autograd.Function over the shifted solve and its adjoint.

`held_out_loss(alpha, beta, op, target, rows, y_rows)` is the mean logistic
loss of the centred held-out scores s_h = (X_h - 1 mu_l^T) w of
w = (B(alpha) + beta I)^{-1} b, differentiable in (alpha, beta):

* forward: one shifted-CG solve at the single shift beta with this call's
  alpha (sda_solve_shifts), the centred ratings (sda_project), the loss;
* backward: sda_adjoint_grad, one adjoint solve on the same symmetric
  operator and two FP64 contractions.

The solve and the adjoint run in libsda's kernels; torch only holds the
device arrays and evaluates the user's loss on the held-out scores.
"""
from __future__ import annotations

import torch

from . import sda


def _solve_opts(op, target: int, tol: float, max_iter: int, alpha: float | None = None):
    o = sda.sda_default_opts()
    o.tol = float(tol)
    o.max_iter = int(max_iter)
    o.target_begin = int(target)
    o.target_count = 1
    o.check_residual = 0
    if alpha is not None:
        o.alpha = float(alpha)
    return o


class HeldOutLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alpha, beta, op, target, rows, y_rows, tol=1e-10, max_iter=20000):
        a, b = float(alpha), float(beta)
        d, n = op.info["n_cols"], op.info["n_rows"]
        w = torch.empty((1, 1, d), dtype=torch.float64, device=rows.device)
        code, rep = sda.sda_solve_shifts(op.handle, [b], _solve_opts(op, target, tol, max_iter, a), w_out=w,
                                         n_report=1)
        scores = torch.empty((1, n), dtype=torch.float64, device=rows.device)
        sda.sda_project(op.handle, w[0, 0], 1, scores, centred=1, target=target)
        s_h = scores[0, rows]
        y = y_rows.to(torch.float64)
        z = -y * s_h
        loss = torch.nn.functional.softplus(z).mean()
        g = (-y * torch.sigmoid(z) / rows.numel()).contiguous()
        ctx.save_for_backward(w, g, rows)
        ctx.op, ctx.target, ctx.a, ctx.b, ctx.tol, ctx.max_iter = op, target, a, b, tol, max_iter
        ctx.iters = rep[0][0]["iters"]
        return loss.detach()

    @staticmethod
    def backward(ctx, grad):
        w, g, rows = ctx.saved_tensors
        code, da, db = sda.sda_adjoint_grad(ctx.op.handle, ctx.target, ctx.a, ctx.b, w[0, 0], g,
                                            rows.to(torch.int64).contiguous(),
                                            _solve_opts(ctx.op, ctx.target, ctx.tol, ctx.max_iter))
        ga = grad * torch.tensor(da, dtype=grad.dtype, device=grad.device)
        gb = grad * torch.tensor(db, dtype=grad.dtype, device=grad.device)
        return ga, gb, None, None, None, None, None, None


def held_out_loss(alpha, beta, op, target, rows, y_rows, tol=1e-10, max_iter=20000):
    """Differentiable held-out logistic loss (see module docstring)."""
    return HeldOutLoss.apply(alpha, beta, op, target, rows, y_rows, tol, max_iter)


class HeldOutLossBatched(torch.autograd.Function):
    """Mean over the targets t0 .. t0 + T - 1 of each one's held-out logistic
    loss at a common (alpha, beta): the forward solves all T targets in the
    batched path (sda_solve_shifts with batch_targets, one shift) and scores
    their held-out rows (sda_project_rows, centred); the backward runs the T
    adjoint solves batched (sda_adjoint_grad_batched) and sums the gradients."""

    @staticmethod
    def forward(ctx, alpha, beta, op, t0, T, rows, row_off, y_rows, tol, max_iter, refine_rounds, refine_tol):
        a, b = float(alpha), float(beta)
        d = op.info["n_cols"]
        dev = rows.device
        w = torch.empty((T, 1, d), dtype=torch.float64, device=dev)
        o = _solve_opts(op, t0, tol, max_iter, a)
        o.target_count, o.batch_targets = int(T), 1
        o.refine_rounds, o.refine_tol = int(refine_rounds), float(refine_tol)
        sda.sda_solve_shifts(op.handle, [b], o, w_out=w, n_report=T)
        off = [int(x) for x in row_off]
        s_h = torch.empty(off[-1], dtype=torch.float64, device=dev)
        for i in range(T):
            r = rows[off[i]:off[i + 1]].contiguous()
            sc = torch.empty((1, r.numel()), dtype=torch.float64, device=dev)
            sda.sda_project_rows(op.handle, w[i, 0], 1, r, sc, centred=1, target=t0 + i)
            s_h[off[i]:off[i + 1]] = sc[0]
        y = y_rows.to(torch.float64)
        z = -y * s_h
        counts = torch.tensor([off[i + 1] - off[i] for i in range(T)], dtype=torch.float64, device=dev)
        per_row = torch.repeat_interleave(1.0 / (counts * T), counts.to(torch.int64))
        loss = (torch.nn.functional.softplus(z) * per_row).sum()
        g = (-y * torch.sigmoid(z) * per_row).contiguous()
        ctx.save_for_backward(w, g, rows)
        ctx.op, ctx.t0, ctx.T, ctx.off, ctx.a, ctx.b = op, t0, T, off, a, b
        ctx.opt = (tol, max_iter, refine_rounds, refine_tol)
        return loss.detach()

    @staticmethod
    def backward(ctx, grad):
        w, g, rows = ctx.saved_tensors
        tol, max_iter, rr, rt = ctx.opt
        o = _solve_opts(ctx.op, ctx.t0, tol, max_iter)
        o.refine_rounds, o.refine_tol = int(rr), float(rt)
        targets = list(range(ctx.t0, ctx.t0 + ctx.T))
        code, da, db, _ = sda.sda_adjoint_grad_batched(ctx.op.handle, targets, ctx.a, [ctx.b] * ctx.T,
                                                       w[:, 0].contiguous(), g, rows.to(torch.int64).contiguous(),
                                                       ctx.off, o)
        ga = grad * torch.tensor(float(da.sum()), dtype=grad.dtype, device=grad.device)
        gb = grad * torch.tensor(float(db.sum()), dtype=grad.dtype, device=grad.device)
        return ga, gb, None, None, None, None, None, None, None, None, None, None


def held_out_loss_batched(alpha, beta, op, t0, T, rows, row_off, y_rows, tol=1e-10, max_iter=20000,
                          refine_rounds=0, refine_tol=float("nan")):
    """Differentiable mean held-out loss of T targets at a common (alpha, beta)
    (see HeldOutLossBatched); rows / y_rows concatenate the targets' held-out
    rows and classes, row_off [T + 1] delimits them."""
    return HeldOutLossBatched.apply(alpha, beta, op, t0, T, rows, row_off, y_rows, tol, max_iter, refine_rounds,
                                    refine_tol)
