"""The held-out selection step (sda_heldout_logistic) against the oracle's
logistic loss: the loss of every (target, shift) and the loss gradient at the
least-loss shift to FP64 rounding, the chosen shift exactly where the least
loss is separated from the next, and valid where it is not.  Covers more
targets than one launch group (256), targets with no rows and with more rows
than a block has threads, an exact tie (the smaller shift), NaN losses (never
least unless all are NaN), and repeated calls (the same bits)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_04794_gb300 import sda

pytestmark = pytest.mark.gpu

NS = 24


def _case(seed=5, T=300):
    rng = np.random.default_rng(seed)
    m = rng.integers(0, 40, T)
    m[[3, 7, 9, 10, T // 3, T - 1]] = [0, 20, 10, 5, 700, 1]
    off = np.concatenate([[0], np.cumsum(m)]).astype(np.int64)
    R = int(off[-1])
    y = np.where(rng.random(R) < 0.3, 1.0, -1.0)
    sc = np.empty(NS * R)
    for t in range(T):
        a, b = off[t], off[t + 1]
        blk = rng.standard_normal((NS, b - a)) * rng.uniform(0.1, 8.0, (NS, 1))
        sc[NS * a:NS * b] = blk.ravel()
    # target 7: shifts 3 and 11 give the same, least loss (identical ratings)
    a, b = off[7], off[8]
    blk = sc[NS * a:NS * b].reshape(NS, b - a)
    blk[3] = 4.0 * y[a:b]
    blk[11] = blk[3]
    # target 9: a NaN rating at shift 0 (its loss is NaN); target 10: every shift NaN
    sc[NS * off[9]] = np.nan
    sc[NS * off[10]:NS * off[11]] = np.nan
    return off, y, sc


def _ref(off, y, sc):
    T = off.size - 1
    loss = np.zeros((T, NS))
    grads = {}
    for t in range(T):
        a, b = off[t], off[t + 1]
        blk = sc[NS * a:NS * b].reshape(NS, b - a)
        for s in range(NS):
            if b > a:
                with np.errstate(over="ignore", invalid="ignore"):
                    loss[t, s], grads[t, s] = oracle.logistic_loss(blk[s], y[a:b])
    return loss, grads


def _run(off, y, sc):
    T, R = off.size - 1, int(off[-1])
    loss = torch.empty((T, NS), dtype=torch.float64, device="cuda")
    best = torch.empty(T, dtype=torch.int32, device="cuda")
    g = torch.empty(R, dtype=torch.float64, device="cuda")
    sda.sda_heldout_logistic(NS, off, torch.from_numpy(sc).cuda(), torch.from_numpy(y).cuda(), loss, best, g)
    torch.cuda.synchronize()
    return loss.cpu().numpy(), best.cpu().numpy(), g.cpu().numpy()


def test_heldout_logistic_matches_oracle():
    off, y, sc = _case()
    loss, best, g = _run(off, y, sc)
    ref, grads = _ref(off, y, sc)
    T = off.size - 1
    fin = np.isfinite(ref)
    assert np.array_equal(np.isnan(loss), np.isnan(ref))
    assert np.all(np.abs(loss[fin] - ref[fin]) <= 1e-14 * np.maximum(1.0, np.abs(ref[fin])))
    for t in range(T):
        a, b = off[t], off[t + 1]
        lt = ref[t]
        if b == a:
            assert best[t] == 0 and np.all(loss[t] == 0.0)
            continue
        if np.all(np.isnan(lt)):
            assert best[t] == 0
        else:
            order = np.argsort(np.where(np.isnan(lt), np.inf, lt), kind="stable")
            least, nxt = lt[order[0]], lt[order[1]]
            if nxt - least > 1e-12 * abs(least):
                assert best[t] == order[0], t
            else:
                assert abs(lt[best[t]] - least) <= 1e-13 * abs(least), t
        gr = grads[t, int(best[t])]
        if np.all(np.isfinite(gr)):
            assert np.all(np.abs(g[a:b] - gr) <= 4e-15 * np.max(np.abs(gr))), t
    assert best[7] == 3                          # exact tie: the smaller shift
    assert not np.isnan(loss[9, best[9]])        # a NaN loss is never least
    assert best[10] == 0                         # every loss NaN


def test_heldout_logistic_repeats_bit_for_bit():
    off, y, sc = _case(seed=6, T=40)
    first = _run(off, y, sc)
    again = _run(off, y, sc)
    for a, b in zip(first, again):
        assert np.array_equal(a, b, equal_nan=True) if a.dtype.kind == "f" else np.array_equal(a, b)
