"""Parity measures of a GPU solution against the FP64 oracle's.

The bar (FP64 oracle, per result): 1e-6 relative on w, AUC equal to 4
decimals (|delta AUC| < 5e-5).  The relative error of any solution w of
(B + beta I) w = b against another w* is bounded by its residuals:

    ||w - w*|| / ||w*|| <= kappa_beta (rho + rho*),
    kappa_beta = (lambda_max(B) + beta) / beta  (B is PSD, so lambda_min >= beta),

rho, rho* the relative FP64 true residuals ||b - (B + beta I) w|| / ||b||.
Where that bound exceeds 1e-6 the 1e-6 bar cannot be asserted for any FP64
solver (the oracle's own error may be that large); there the error is
reported beside its bound and only checked against the bound.  The
element-wise error max_j |w_j - w*_j| / max_j |w*_j| is checked at the same
bar, so that a few wrong entries (rare features) cannot hide under a norm.
"""
from __future__ import annotations

import numpy as np

import oracle

W_BAR = 1e-6
AUC_BAR = 5e-5


def lambda_max(o: "oracle.Oracle", iters: int = 60, seed: int = 0) -> float:
    """Upper estimate of lambda_max(B): power iteration on the oracle's operator
    (its Rayleigh quotient approaches lambda_max from below), with 10 % margin."""
    x = np.random.default_rng(seed).standard_normal(o.d)
    lam = 0.0
    for _ in range(iters):
        x /= np.linalg.norm(x)
        y = o.apply(x, 0.0)
        lam = float(x @ y)
        x = y
    return 1.1 * lam


def compare(w: np.ndarray, w_ref: np.ndarray, beta: float, lam_max: float, rho: float, rho_ref: float) -> dict:
    """Errors of w against w_ref and the residual bound of the norm-wise error."""
    ref_inf = float(np.max(np.abs(w_ref)))
    diff = w - w_ref
    rel = float(np.linalg.norm(diff) / max(np.linalg.norm(w_ref), 1e-300))
    elem = float(np.max(np.abs(diff)) / max(ref_inf, 1e-300))
    kappa = (lam_max + beta) / beta
    bound = kappa * (abs(rho) + abs(rho_ref))
    return {"beta": float(beta), "rel": rel, "elem": elem, "kappa": kappa, "bound": bound,
            "asserted": bound <= W_BAR}


def check(res: dict, where=""):
    """1e-6 norm-wise and element-wise where the bound permits it; else the
    norm-wise error within its bound (a larger error means a wrong solution)."""
    if res["asserted"]:
        assert res["rel"] <= W_BAR and res["elem"] <= W_BAR, (where, res)
    else:
        assert res["rel"] <= max(res["bound"], W_BAR), (where, res)
        print("w error beside its bound (1e-6 not attainable at this shift):", where, res)


def auc_of(X_rows_times_w: np.ndarray, truth: np.ndarray) -> float:
    return oracle.auc(X_rows_times_w, truth)
