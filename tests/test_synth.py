"""The seeded input generator: determinism, shapes, and the kNN graph (Sec. 2.4)."""
import numpy as np

from paper_1709_04794_gb300 import synth


def _bruteforce_knn(prob, k):
    n, d = prob.n, prob.d
    A = np.zeros((n, d), dtype=np.float64)
    A[np.repeat(np.arange(n), np.diff(prob.x_ptr)), prob.x_col] = 1.0
    inter = A @ A.T
    sz = A.sum(axis=1)
    jac = inter / (sz[:, None] + sz[None, :] - inter)
    np.fill_diagonal(jac, -1.0)
    nbr = -np.ones((n, k), dtype=np.int64)
    sim = np.zeros((n, k))
    for i in range(n):
        # rank by (similarity desc, index asc); similarity 0 never makes an edge
        order = np.lexsort((np.arange(n), -jac[i]))
        m = 0
        for j in order[:k]:
            if jac[i, j] > 0:
                nbr[i, m], sim[i, m] = j, jac[i, j]
                m += 1
    return nbr, sim


def test_knn_graph_equals_bruteforce(cfg1):
    nbr, sim = _bruteforce_knn(cfg1, cfg1.workload.knn_k)
    sp, sc, sv = synth.union_graph(nbr, sim)
    assert np.array_equal(sp, cfg1.s_ptr)
    assert np.array_equal(sc, cfg1.s_col)
    assert np.array_equal(sv, cfg1.s_val)


def test_graph_symmetric_zero_diagonal_laplacian_psd(cfg1):
    n = cfg1.n
    S = np.zeros((n, n))
    S[np.repeat(np.arange(n), np.diff(cfg1.s_ptr)), cfg1.s_col] = cfg1.s_val
    assert np.array_equal(S, S.T)
    assert np.all(np.diag(S) == 0)
    assert np.all((cfg1.s_val > 0) & (cfg1.s_val <= 1))
    L = np.diag(S.sum(axis=1)) - S
    assert np.allclose(L @ np.ones(n), 0, atol=1e-12)       # L 1 = 0 (Sec. 2.5.2)
    assert np.linalg.eigvalsh(L).min() > -1e-10


def test_candidate_knn_with_full_cap_is_exact():
    p = synth.custom_problem(300, 500, 12, seed=3, k=6)
    nbr_exact, sim_exact = synth.knn_lists(p.x_ptr, p.x_col, p.d, 6, None)
    nbr_cap, sim_cap = synth.knn_lists(p.x_ptr, p.x_col, p.d, 6, p.n)
    assert np.array_equal(nbr_exact, nbr_cap)
    # a finite cap gives a subset-of-candidates approximation of the same shape
    nbr_c, sim_c = synth.knn_lists(p.x_ptr, p.x_col, p.d, 6, 8)
    assert nbr_c.shape == nbr_exact.shape
    assert np.all(sim_c <= sim_exact[:, :1] + 1e-15)


def test_knn_thread_count_independent():
    p = synth.custom_problem(400, 300, 10, seed=4, k=5)
    a = synth.knn_lists(p.x_ptr, p.x_col, p.d, 5, 30, threads=1)
    b = synth.knn_lists(p.x_ptr, p.x_col, p.d, 5, 30, threads=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_workload_shape(cfg1):
    wl = cfg1.workload
    assert cfg1.n == 2000 and cfg1.d == 4096
    rows = np.diff(cfg1.x_ptr)
    assert rows.min() >= 1 and abs(rows.mean() - 40) < 1.5
    for i in range(0, cfg1.n, 97):                          # distinct sorted columns per row
        c = cfg1.x_col[cfg1.x_ptr[i]:cfg1.x_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    y = cfg1.labels[0]
    assert (y != 0).sum() == 200 and (y > 0).sum() == 60
    h = cfg1.heldout[0]
    assert np.all(y[h] == 0) and h.size == 50
    assert np.all(cfg1.truth[0][y != 0] == y[y != 0])
    assert len(cfg1.shifts) == 10 and np.isclose(cfg1.shifts[0], 1e-4)
    # Zipf popularity: the most common feature is in most rows
    cnt = np.bincount(cfg1.x_col, minlength=cfg1.d)
    assert cnt.max() > 0.9 * cfg1.n
    assert wl.alpha == 0.1


def test_deterministic():
    a = synth.custom_problem(200, 100, 6, seed=21, values="counts")
    b = synth.custom_problem(200, 100, 6, seed=21, values="counts")
    for f in ("x_ptr", "x_col", "x_val", "s_ptr", "s_col", "s_val", "labels"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert set(np.unique(a.x_val)) <= set(range(1, 9))
