"""Seeded synthetic inputs shaped like the paper's workloads.

The paper measures on ECFP fingerprint matrices (ChEMBL: 167,668 x 291,714,
12.2M nonzeros, density 0.025 %, Table 3; Janssen: ~2M compounds, >10M
features, Sec. 5.2).  Neither data set is available, so seeded stand-ins with
the same structure are generated here:

* X (N x D, CSR): nonzeros per row ~ Poisson(mean), clipped to >= 1; the
  columns of a row are drawn without replacement from a Zipf(s) popularity
  law over a seeded permutation of the feature ids (fingerprint bits have a
  few very common and a long tail of rare substructures).  Values are binary
  1, or counts 1..8 from a geometric law (p = 0.7) truncated to 1..8.
* S (N x N, CSR, symmetric, zero diagonal): the union of the directed
  k-nearest-neighbour lists under the Jaccard (= Tanimoto on binary
  supports) similarity, with the similarity as edge weight (Sec. 2.4,
  Tanimoto kNN in Sec. 5.1).  Exact for small N; for large N the
  candidates of a row are the rows that share one of its rarer features.
* labels: one int8 vector per binary target, +1 / -1 on the labelled rows,
  0 elsewhere.  Classes come from a planted sparse linear model (1 % of the
  features informative, drawn among the 20 % most frequent, Gaussian
  weights, Gaussian score noise at half the score's spread); the
  labelled subset is uniform, with the exact positive share requested.
  A disjoint held-out set of unlabelled rows keeps its true labels for AUC.

The two largest workloads (500,000 and 2,000,000 rows, 64 and 1,000
targets) are drawn by the native helpers of synth_native.c with the same
laws: one counter-based random stream per row of X and per target, so that
they take seconds on many cores; their score spread is measured over each
target's labelled and held-out rows (the only rows whose scores are drawn),
and their `truth` holds the classes of those rows only (0 elsewhere).

This module holds none of the solver's arithmetic: no means, no Laplacian,
no operator.  Both the oracle and the CUDA path consume its arrays.
"""
from __future__ import annotations

import ctypes
import functools
import os
from dataclasses import dataclass, field

import numpy as np

from . import _build

# --------------------------------------------------------------------------
# Workloads (sizes of the paper-shaped synthetic problems)
# --------------------------------------------------------------------------


@dataclass(frozen=True)
class Workload:
    name: str
    n: int                      # samples (rows of X)
    d: int                      # features (columns of X)
    nnz_mean: float             # Poisson mean of nonzeros per row
    values: str                 # "binary" | "counts"
    n_targets: int
    labelled: tuple             # ("fixed", ell) | ("frac", f) | ("loguniform", lo, hi)
    pos_frac: tuple             # ("fixed", q) | ("uniform", lo, hi) | ("lognormal_median", m)
    knn_k: int
    alpha: float
    shifts: tuple               # (lo, hi, count), log-spaced
    seed: int
    value_dtype: str            # storage dtype of X on the device in the mixed path
    zipf_s: float = 1.1
    knn_cap: int | None = None  # None: exact kNN
    holdout_ratio: float = 0.25  # held-out rows per labelled row (20 % of all known labels)
    generator: str = "numpy"    # "numpy" | "native" (synth_native.c, the large workloads)

    def shift_values(self) -> np.ndarray:
        lo, hi, cnt = self.shifts
        return np.logspace(np.log10(lo), np.log10(hi), int(cnt))


WORKLOADS = {
    "single_fp64_2k": Workload(
        name="single_fp64_2k", n=2000, d=4096, nnz_mean=40, values="binary", n_targets=1,
        labelled=("fixed", 200), pos_frac=("fixed", 0.30), knn_k=10, alpha=0.1,
        shifts=(1e-4, 1e2, 10), seed=17090001, value_dtype="f64"),
    "single_mixed_200k": Workload(
        name="single_mixed_200k", n=200_000, d=131_072, nnz_mean=60, values="counts", n_targets=1,
        labelled=("frac", 0.05), pos_frac=("fixed", 0.10), knn_k=10, alpha=0.1,
        shifts=(1e-5, 1e3, 32), seed=17090002, value_dtype="f16", knn_cap=96),
    "batched_256t_200k": Workload(
        name="batched_256t_200k", n=200_000, d=131_072, nnz_mean=60, values="counts", n_targets=256,
        labelled=("loguniform", 100, 20_000), pos_frac=("uniform", 0.01, 0.50), knn_k=10,
        alpha=0.1, shifts=(1e-5, 1e3, 16), seed=17090002, value_dtype="f16", knn_cap=96),
    "adjoint_64t_500k": Workload(
        name="adjoint_64t_500k", n=500_000, d=262_144, nnz_mean=50, values="binary", n_targets=64,
        labelled=("loguniform", 100, 20_000), pos_frac=("uniform", 0.01, 0.50), knn_k=10,
        alpha=0.1, shifts=(1e-5, 1e3, 16), seed=17090004, value_dtype="f8e4m3", knn_cap=96,
        generator="native"),
    "large_1000t_2m": Workload(
        name="large_1000t_2m", n=2_000_000, d=1_048_576, nnz_mean=45, values="binary",
        n_targets=1000, labelled=("loguniform", 50, 50_000), pos_frac=("lognormal_median", 0.02),
        knn_k=8, alpha=0.1, shifts=(1e-5, 1e3, 24), seed=17090005, value_dtype="f8e4m3",
        knn_cap=96, generator="native"),
}


# --------------------------------------------------------------------------
# X
# --------------------------------------------------------------------------


def zipf_csr(rng: np.random.Generator, n: int, d: int, nnz_mean: float, s: float):
    """Rows with Poisson(nnz_mean) nonzeros (>= 1) at Zipf(s)-popular features.

    Within a row the features are distinct: draws are taken with
    replacement and the first occurrences kept in draw order, topping up
    rows that came out short.  Returns (row_ptr int64, col int32), columns
    sorted within each row."""
    counts = rng.poisson(nnz_mean, size=n).astype(np.int64)
    counts = np.clip(counts, 1, max(1, d // 2))
    w = np.arange(1, d + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    perm = rng.permutation(d).astype(np.int64)  # popularity rank -> feature id

    have_keys = np.empty(0, dtype=np.int64)     # row * d + feature, kept so far
    short = np.arange(n, dtype=np.int64)
    need = counts.copy()
    while short.size:
        m = (need[short] * 3) // 2 + 8
        rows = np.repeat(short, m)
        u = rng.random(rows.size)
        rank = np.minimum(np.searchsorted(cdf, u, side="right"), d - 1)
        keys = rows * d + perm[rank]
        allk = np.concatenate([have_keys, keys])
        _, first = np.unique(allk, return_index=True)
        first.sort()
        kept = allk[first]
        krow = kept // d
        # position of each kept key within its row (kept is row-grouped after the sort below)
        order = np.argsort(krow, kind="stable")
        kept = kept[order]
        krow = krow[order]
        starts = np.searchsorted(krow, np.arange(n), side="left")
        pos = np.arange(kept.size) - starts[krow]
        sel = pos < counts[krow]
        have_keys = kept[sel]
        got = np.bincount(krow[sel], minlength=n)
        need = counts - got
        short = np.nonzero(need > 0)[0]
    have_keys.sort()
    row = have_keys // d
    col = (have_keys % d).astype(np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(row, minlength=n), out=row_ptr[1:])
    return row_ptr, col


def count_values(rng: np.random.Generator, nnz: int, p: float = 0.7, vmax: int = 8) -> np.ndarray:
    """Counts 1..vmax with P(v) proportional to p (1-p)^(v-1) (exact in FP16 and FP8 e4m3)."""
    v = np.arange(1, vmax + 1)
    pmf = p * (1 - p) ** (v - 1)
    cdf = np.cumsum(pmf) / pmf.sum()
    return (np.minimum(np.searchsorted(cdf, rng.random(nnz), side="right"), vmax - 1) + 1).astype(np.float64)


# --------------------------------------------------------------------------
# S: kNN graph, Jaccard weights
# --------------------------------------------------------------------------


@functools.lru_cache(maxsize=1)
def _knn_lib():
    lib = ctypes.CDLL(_build.build_synth())
    vp, i64, i32, f64, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64
    for name, args in (("synth_knn_jaccard", [i64, i64, vp, vp, i32, i64, vp, vp, i32]),
                       ("synth_row_counts", [i64, i64, f64, u64, vp, i32]),
                       ("synth_fill_rows", [i64, i64, vp, vp, i32, vp, u64, vp, vp, vp, i32]),
                       ("synth_planted", [i64, i64, vp, vp, vp, i32, vp, vp, vp, i64, i64, f64, u64, vp, vp,
                                          vp, i64, vp, i32])):
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        fn.argtypes = args
    return lib


def knn_lists(row_ptr, col, d: int, k: int, cap: int | None = None, threads: int = 0):
    """Directed kNN lists (n x k neighbour ids, -1 padded; n x k similarities)."""
    n = row_ptr.size - 1
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    nbr = np.empty((n, k), dtype=np.int32)
    sim = np.empty((n, k), dtype=np.float64)
    rc = _knn_lib().synth_knn_jaccard(n, d, row_ptr.ctypes.data, col.ctypes.data, k,
                                      n if cap is None else int(cap), nbr.ctypes.data,
                                      sim.ctypes.data, int(threads))
    if rc != 0:
        raise RuntimeError("synth_knn_jaccard failed with code %d" % rc)
    return nbr, sim


def union_graph(nbr: np.ndarray, sim: np.ndarray):
    """Symmetric CSR (row_ptr int64, col int32, weight float64) of the union of directed lists."""
    n, k = nbr.shape
    src = np.repeat(np.arange(n, dtype=np.int64), k)
    dst = nbr.reshape(-1).astype(np.int64)
    wt = sim.reshape(-1)
    ok = dst >= 0
    src, dst, wt = src[ok], dst[ok], wt[ok]
    a = np.concatenate([src, dst])
    b = np.concatenate([dst, src])
    w = np.concatenate([wt, wt])
    key = a * n + b
    key, first = np.unique(key, return_index=True)
    w = w[first]
    a = key // n
    b = (key % n).astype(np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(a, minlength=n), out=row_ptr[1:])
    return row_ptr, b, w


# --------------------------------------------------------------------------
# Labels
# --------------------------------------------------------------------------


def planted_target(rng, x_ptr, x_col, x_val, d: int, n_labelled: int, pos_frac: float,
                   holdout_ratio: float):
    """One binary target: (labels int8 [N], truth int8 [N], held-out row ids int64)."""
    n = x_ptr.size - 1
    n_inf = max(1, int(round(0.01 * d)))
    # informative features among the 20 % most frequent ones, so that every row sees a few
    freq = np.bincount(x_col, minlength=d)
    pool = np.argsort(-freq, kind="stable")[:max(n_inf, d // 5)]
    wstar = np.zeros(d)
    wstar[rng.choice(pool, size=n_inf, replace=False)] = rng.standard_normal(n_inf)
    row = np.repeat(np.arange(n), np.diff(x_ptr))
    z = np.bincount(row, weights=x_val * wstar[x_col], minlength=n)
    sd = z.std()
    score = z + rng.standard_normal(n) * 0.5 * (sd if sd > 0 else 1.0)
    n_labelled = int(min(max(n_labelled, 2), n))
    lab = rng.choice(n, size=n_labelled, replace=False)
    n_pos = int(min(max(1, round(pos_frac * n_labelled)), n_labelled - 1))
    order = lab[np.argsort(-score[lab], kind="stable")]
    pos, neg = order[:n_pos], order[n_pos:]
    thresh = 0.5 * (score[pos].min() + score[neg].max())
    truth = np.where(score > thresh, 1, -1).astype(np.int8)
    truth[pos] = 1
    truth[neg] = -1
    y = np.zeros(n, dtype=np.int8)
    y[pos] = 1
    y[neg] = -1
    unl = np.nonzero(y == 0)[0]
    h = int(min(unl.size, max(1, int(np.ceil(holdout_ratio * n_labelled)))))
    held = np.sort(rng.choice(unl, size=h, replace=False)).astype(np.int64)
    return y, truth, held


def _draw_sizes(rng, wl: Workload):
    t = wl.n_targets
    kind = wl.labelled[0]
    if kind == "fixed":
        ell = np.full(t, wl.labelled[1], dtype=np.int64)
    elif kind == "frac":
        ell = np.full(t, int(round(wl.labelled[1] * wl.n)), dtype=np.int64)
    else:
        lo, hi = wl.labelled[1], wl.labelled[2]
        ell = np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), size=t))).astype(np.int64)
    kind = wl.pos_frac[0]
    if kind == "fixed":
        q = np.full(t, wl.pos_frac[1])
    elif kind == "uniform":
        q = rng.uniform(wl.pos_frac[1], wl.pos_frac[2], size=t)
    else:
        q = np.clip(wl.pos_frac[1] * np.exp(0.8 * rng.standard_normal(t)), 0.002, 0.5)
    return ell, q


# --------------------------------------------------------------------------
# Whole problems
# --------------------------------------------------------------------------


@dataclass
class Problem:
    workload: Workload
    x_ptr: np.ndarray
    x_col: np.ndarray
    x_val: np.ndarray          # float64, exact small integers
    s_ptr: np.ndarray
    s_col: np.ndarray
    s_val: np.ndarray          # float64 Jaccard weights
    labels: np.ndarray         # int8 [T, N]
    truth: np.ndarray          # int8 [T, N]
    heldout: list = field(default_factory=list)   # per target, int64 row ids
    shifts: np.ndarray = None
    alpha: float = 0.1

    @property
    def n(self):
        return self.x_ptr.size - 1

    @property
    def d(self):
        return self.workload.d


def _zipf_cdf(d: int, s: float) -> np.ndarray:
    w = np.arange(1, d + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    cdf[-1] = 1.0
    return cdf


def _geometric_cdf(p: float = 0.7, vmax: int = 8) -> np.ndarray:
    v = np.arange(1, vmax + 1)
    pmf = p * (1 - p) ** (v - 1)
    cdf = np.cumsum(pmf) / pmf.sum()
    cdf[-1] = 1.0
    return cdf


def native_x(wl: Workload, rng: np.random.Generator):
    """X of a large workload from synth_native.c: the same laws as zipf_csr and
    count_values, one random stream per row (seeded from `rng`)."""
    lib = _knn_lib()
    seed = int(rng.integers(0, 2**63 - 1))
    perm = rng.permutation(wl.d).astype(np.int64)
    cdf = _zipf_cdf(wl.d, wl.zipf_s)
    counts = np.empty(wl.n, dtype=np.int64)
    if lib.synth_row_counts(wl.n, wl.d, float(wl.nnz_mean), seed, counts.ctypes.data, 0) != 0:
        raise RuntimeError("synth_row_counts failed")
    x_ptr = np.zeros(wl.n + 1, dtype=np.int64)
    np.cumsum(counts, out=x_ptr[1:])
    x_col = np.empty(int(x_ptr[-1]), dtype=np.int32)
    x_val = np.empty(int(x_ptr[-1]), dtype=np.float64)
    vcdf = _geometric_cdf()
    rc = lib.synth_fill_rows(wl.n, wl.d, cdf.ctypes.data, perm.ctypes.data, 0 if wl.values == "binary" else 1,
                             vcdf.ctypes.data, seed, x_ptr.ctypes.data, x_col.ctypes.data, x_val.ctypes.data, 0)
    if rc != 0:
        raise RuntimeError("synth_fill_rows failed with code %d" % rc)
    return x_ptr, x_col, x_val


def make_x(wl: Workload, rng: np.random.Generator):
    if wl.generator == "native":
        return native_x(wl, rng)
    x_ptr, x_col = zipf_csr(rng, wl.n, wl.d, wl.nnz_mean, wl.zipf_s)
    if wl.values == "binary":
        x_val = np.ones(x_col.size)
    else:
        x_val = count_values(rng, x_col.size)
    return x_ptr, x_col, x_val


def native_targets(wl: Workload, trng: np.random.Generator, x_ptr, x_col, x_val, t: int):
    """Planted targets of a large workload from synth_native.c (the law of
    planted_target, one random stream per target)."""
    ell, q = _draw_sizes(trng, wl)
    ell, q = np.ascontiguousarray(ell[:t], dtype=np.int64), np.ascontiguousarray(q[:t], dtype=np.float64)
    n, d = wl.n, wl.d
    n_inf = max(1, int(round(0.01 * d)))
    freq = np.bincount(x_col, minlength=d)
    pool = np.ascontiguousarray(np.argsort(-freq, kind="stable")[:max(n_inf, d // 5)], dtype=np.int32)
    seed = int(trng.integers(0, 2**63 - 1))
    hmax = int(max(1, np.ceil(wl.holdout_ratio * max(int(ell.max()) if t else 2, 2))))
    labels = np.zeros((t, n), dtype=np.int8)
    truth = np.zeros((t, n), dtype=np.int8)
    held = np.zeros((t, hmax), dtype=np.int64)
    nheld = np.zeros(t, dtype=np.int64)
    rc = _knn_lib().synth_planted(n, d, x_ptr.ctypes.data, x_col.ctypes.data, x_val.ctypes.data, t,
                                  ell.ctypes.data, q.ctypes.data, pool.ctypes.data, pool.size, n_inf,
                                  float(wl.holdout_ratio), seed, labels.ctypes.data, truth.ctypes.data,
                                  held.ctypes.data, hmax, nheld.ctypes.data, 0)
    if rc != 0:
        raise RuntimeError("synth_planted failed with code %d" % rc)
    return labels, truth, [held[i, :nheld[i]].copy() for i in range(t)]


@functools.lru_cache(maxsize=4)
def make_problem(name: str, n_targets: int | None = None) -> Problem:
    """Deterministic problem for a named workload (optionally fewer targets)."""
    wl = WORKLOADS[name]
    rng = np.random.default_rng(wl.seed)
    x_ptr, x_col, x_val = make_x(wl, rng)
    nbr, sim = knn_lists(x_ptr, x_col, wl.d, wl.knn_k, wl.knn_cap)
    s_ptr, s_col, s_val = union_graph(nbr, sim)
    t = wl.n_targets if n_targets is None else int(n_targets)
    trng = np.random.default_rng(wl.seed + 7)
    if wl.generator == "native":
        labels, truth, held = native_targets(wl, trng, x_ptr, x_col, x_val, t)
        return Problem(wl, x_ptr, x_col, x_val, s_ptr, s_col, s_val, labels, truth, held,
                       wl.shift_values(), wl.alpha)
    ell, q = _draw_sizes(trng, wl)
    labels = np.zeros((t, wl.n), dtype=np.int8)
    truth = np.zeros((t, wl.n), dtype=np.int8)
    held = []
    for i in range(t):
        y, tr, h = planted_target(trng, x_ptr, x_col, x_val, wl.d, int(ell[i]), float(q[i]),
                                  wl.holdout_ratio)
        labels[i], truth[i] = y, tr
        held.append(h)
    return Problem(wl, x_ptr, x_col, x_val, s_ptr, s_col, s_val, labels, truth, held,
                   wl.shift_values(), wl.alpha)


def custom_problem(n: int, d: int, nnz_mean: float, seed: int, *, values: str = "binary",
                   n_targets: int = 1, n_labelled: int = 40, pos_frac: float = 0.3, k: int = 5,
                   alpha: float = 0.1, shifts=(1e-3, 1e1, 5), zipf_s: float = 1.1,
                   knn_cap: int | None = None) -> Problem:
    """Small seeded problem of any shape (tests: ragged tiles, edge cases)."""
    wl = Workload(name="custom", n=n, d=d, nnz_mean=nnz_mean, values=values, n_targets=n_targets,
                  labelled=("fixed", n_labelled), pos_frac=("fixed", pos_frac), knn_k=k,
                  alpha=alpha, shifts=tuple(shifts), seed=seed, value_dtype="f64", zipf_s=zipf_s,
                  knn_cap=knn_cap)
    rng = np.random.default_rng(seed)
    x_ptr, x_col, x_val = make_x(wl, rng)
    nbr, sim = knn_lists(x_ptr, x_col, d, k, knn_cap)
    s_ptr, s_col, s_val = union_graph(nbr, sim)
    labels = np.zeros((n_targets, n), dtype=np.int8)
    truth = np.zeros((n_targets, n), dtype=np.int8)
    held = []
    for i in range(n_targets):
        y, tr, h = planted_target(rng, x_ptr, x_col, x_val, d, n_labelled, pos_frac, 0.25)
        labels[i], truth[i] = y, tr
        held.append(h)
    return Problem(wl, x_ptr, x_col, x_val, s_ptr, s_col, s_val, labels, truth, held,
                   wl.shift_values(), alpha)


def random_r(seed: int, d: int) -> np.ndarray:
    """The random start vector r ~ U(-1, 1)^D of Algorithm 7 (passed in as an input)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=d)
