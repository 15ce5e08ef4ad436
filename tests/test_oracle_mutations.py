"""Planted mistakes in copies of the C oracle must fail at least one pin.

Each mutation is a plausible slip (a dropped term, a wrong sign or index,
swapped weights).  The mutated source is compiled to a temporary library on
the CPU and run through the pin checks below; the real oracle is untouched.
"""
import os
import tempfile

import numpy as np
import pytest
import scipy.linalg

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "sda_oracle.c")

MUTATIONS = {
    # Alg. 3 printed index slip: alpha_i instead of alpha_{i+1}
    "alpha_index_slip": ("as[s] = alpha_new * ratio * ratio;", "as[s] = alpha * ratio * ratio;"),
    # drop the rank-1 centring correction of Sec. 3.2.3
    "no_centring": ("q[j] = q[j] - P->mu[j] * sum_v + sigma * p[j];", "q[j] = q[j] + sigma * p[j];"),
    # wrong sign in the Laplacian L = D - S
    "laplacian_sign": ("double lu = P->deg[i] * u[i] - su;", "double lu = P->deg[i] * u[i] + su;"),
    # swapped weights of the two terms of eq. (7)
    "swapped_weights": ("v[i] = P->omega * pu + P->alpha * lu;", "v[i] = P->alpha * pu + P->omega * lu;"),
    # sign slip in the zeta recurrence of Alg. 3
    "zeta_sign": ("(1.0 - delta * gamma)", "(1.0 + delta * gamma)"),
    # mean not divided by l (Alg. 7 step 3)
    "mean_unscaled": ("P->mu[j] /= ell;", "P->mu[j] /= 1.0;"),
    # transposed operand: X^T v read through the CSR row pointers
    "transposed_xt": ("for (int64_t e = P->tp[j]; e < P->tp[j + 1]; ++e) s += P->tv[e] * v[P->tr[e]];",
                      "for (int64_t e = P->tp[j]; e < P->tp[j + 1]; ++e) s += P->tv[e] * v[P->tr[e] % (int32_t)(P->d)];"),
    # shift update of W uses the base gamma instead of gamma^b
    "shift_gamma": ("W[(int64_t)s * d + j] -= gs[s] * Ps[(int64_t)s * d + j];",
                    "W[(int64_t)s * d + j] -= gamma * Ps[(int64_t)s * d + j];"),
}


def _pins_pass(so, tiny, cfg1):
    """The subset of pins that runs in a second: returns True if all hold."""
    X = oracle.dense_x(tiny.x_ptr, tiny.x_col, tiny.x_val, tiny.d)
    y = tiny.labels[0]
    o = oracle.Oracle(tiny.x_ptr, tiny.x_col, tiny.x_val, tiny.s_ptr, tiny.s_col, tiny.s_val, y,
                      tiny.d, tiny.alpha, so_path=so)
    B = oracle.dense_operator(X, tiny.s_ptr, tiny.s_col, tiny.s_val, y, tiny.alpha)
    p = np.random.default_rng(0).standard_normal(tiny.d)
    if np.linalg.norm(o.apply(p, 0.3) - (B @ p + 0.3 * p)) > 1e-10 * np.linalg.norm(B @ p):
        return False
    mu, mp, mn, _ = o.class_means()
    if not np.allclose(mu, X[y != 0].mean(axis=0), atol=1e-13):
        return False
    b = mp - mn
    res = o.shifted_cg(b, tiny.shifts, tol=1e-13, max_iter=3000)
    for s, beta in enumerate(tiny.shifts):
        w = scipy.linalg.solve(B + beta * np.eye(tiny.d), b, assume_a="pos")
        if np.linalg.norm(res.W[s] - w) > 1e-8 * np.linalg.norm(w):
            return False
    oc = oracle.Oracle(cfg1.x_ptr, cfg1.x_col, cfg1.x_val, cfg1.s_ptr, cfg1.s_col, cfg1.s_val,
                       cfg1.labels[0], cfg1.d, cfg1.alpha, so_path=so)
    bc = oc.rhs_canonical()
    r5 = oc.shifted_cg(bc, cfg1.shifts, fixed_iters=5)
    for s, beta in enumerate(cfg1.shifts):
        w, *_ = oc.cg(bc, beta, fixed_iters=5)
        if np.linalg.norm(r5.W[s] - w) > 1e-10 * np.linalg.norm(w):
            return False
    return True


def test_unmutated_oracle_passes(tiny, cfg1):
    assert _pins_pass(oracle.build(), tiny, cfg1)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tiny, cfg1):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found: " + name
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "mut.c")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        so = os.path.join(tmp, "mut.so")
        import subprocess
        r = subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", path, "-o", so,
                            "-lm"], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        assert not _pins_pass(so, tiny, cfg1), "pins did not catch " + name


# A mistake in the regression operator built on the same code (CSR-SDA,
# Algorithm 5, line 5): keeping the centring must fail the X^T X pin.  (SA-SDA
# runs the unchanged operator with X = I, covered by the mutations above.)
MODE_MUTATIONS = {
    "regression_keeps_centring": ("if (P) memset(P->mu, 0, (size_t)(d > 0 ? d : 1) * sizeof(double));",
                                  "(void)P;"),
}


def _regression_pin_passes(so):
    from paper_1709_04794_gb300 import synth
    p = synth.custom_problem(120, 30, 6, seed=19, values="counts")
    o = oracle.Oracle.regression(p.x_ptr, p.x_col, p.x_val, p.d, so_path=so)
    X = oracle.dense_x(p.x_ptr, p.x_col, p.x_val, p.d)
    x = np.random.default_rng(3).standard_normal(p.d)
    ref = X.T @ (X @ x) + 0.7 * x
    return bool(np.linalg.norm(o.apply(x, 0.7) - ref) <= 1e-12 * np.linalg.norm(ref))


def _compile_mutant(tmp, old, new):
    import subprocess
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found"
    path = os.path.join(tmp, "mut.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(tmp, "mut.so")
    r = subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", path, "-o", so, "-lm"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return so


def test_unmutated_regression_pin_passes():
    assert _regression_pin_passes(oracle.build())


@pytest.mark.parametrize("name", sorted(MODE_MUTATIONS))
def test_planted_mode_mistake_is_caught(name):
    old, new = MODE_MUTATIONS[name]
    with tempfile.TemporaryDirectory() as tmp:
        so = _compile_mutant(tmp, old, new)
        assert not _regression_pin_passes(so), "pin did not catch " + name
