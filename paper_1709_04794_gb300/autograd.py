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
