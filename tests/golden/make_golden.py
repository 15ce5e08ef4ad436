"""Writes the stored expected values of tests/test_golden.py.

Inputs: a small seeded problem from the shared generator (300 samples x 96
count features, kNN graph k = 5, one target with 80 labelled samples, four
shifts 1e-1..1e2, alpha 0.1, scatter weight 1 - alpha as in eq. 7), stored
with the results so that they do not depend on the generator's host library.
Outputs: the FP64 oracle's shifted-CG solutions (Algorithm 3, base shift the
smallest, relative tolerance 1e-13), its iteration counts, and the AUC of the
scores X w on the held-out rows (Sec. 5.1); and, in a second file, the
solutions of the same sweep for CSR-SDA's regression operator X^T X (b = X^T z,
z seeded) and for SA-SDA's operator (X = I_N).  Only oracle/ computes them.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1709_04794_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "small_300x96_fp64.json")
OUT_MODES = os.path.join(HERE, "small_300x96_modes_fp64.json")


def main():
    p = synth.custom_problem(300, 96, 10, seed=1709, values="counts", n_labelled=80, k=5,
                             shifts=(1e-1, 1e2, 4))
    o = oracle.from_problem(p)
    b = o.rhs_canonical()
    res = o.shifted_cg(b, p.shifts, tol=1e-13, max_iter=50000)
    assert res.status == 0
    X = oracle.dense_x(p.x_ptr, p.x_col, p.x_val, p.d)
    rows = np.asarray(p.heldout[0])
    aucs = [oracle.auc(X[rows] @ res.W[s], p.truth[0][rows]) for s in range(len(p.shifts))]
    doc = {
        "source": "tests/golden/make_golden.py (FP64 oracle, Algorithm 3, tol 1e-13)",
        "n": int(p.n), "d": int(p.d), "alpha": float(p.alpha),
        "x_ptr": p.x_ptr.tolist(), "x_col": p.x_col.tolist(), "x_val": p.x_val.tolist(),
        "s_ptr": p.s_ptr.tolist(), "s_col": p.s_col.tolist(), "s_val": p.s_val.tolist(),
        "labels": p.labels[0].tolist(), "truth": p.truth[0].tolist(), "heldout": rows.tolist(),
        "shifts": [float(x) for x in p.shifts],
        "rhs": b.tolist(),
        "w": res.W.tolist(), "iters": res.iters.tolist(), "auc": aucs,
    }
    with open(OUT, "w") as f:
        json.dump(doc, f)
    print("wrote", OUT)
    # the same X and graph under the two other operators: CSR-SDA's regression
    # step (Algorithm 5, line 5: X^T X, b = X^T z) and SA-SDA (Algorithm 6: X = I_N)
    z = np.random.default_rng(17090).uniform(-1.0, 1.0, p.n)
    rows_all = np.repeat(np.arange(p.n), np.diff(p.x_ptr))
    breg = np.bincount(p.x_col, weights=p.x_val * z[rows_all], minlength=p.d)
    oreg = oracle.Oracle.regression(p.x_ptr, p.x_col, p.x_val, p.d)
    rreg = oreg.shifted_cg(breg, p.shifts, tol=1e-13, max_iter=50000)
    assert rreg.status == 0
    n = p.n
    osa = oracle.Oracle(np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n),
                        p.s_ptr, p.s_col, p.s_val, p.labels[0], n, p.alpha)
    bsa = osa.rhs_canonical()
    rsa = osa.shifted_cg(bsa, p.shifts, tol=1e-13, max_iter=50000)
    assert rsa.status == 0
    modes = {
        "source": "tests/golden/make_golden.py (FP64 oracle, Algorithm 3, tol 1e-13)",
        "inputs": os.path.basename(OUT),
        "regression": {"z": z.tolist(), "rhs": breg.tolist(), "w": rreg.W.tolist(), "iters": rreg.iters.tolist()},
        "sa": {"rhs": bsa.tolist(), "z": rsa.W.tolist(), "iters": rsa.iters.tolist()},
    }
    with open(OUT_MODES, "w") as f:
        json.dump(modes, f)
    print("wrote", OUT_MODES)


if __name__ == "__main__":
    main()
