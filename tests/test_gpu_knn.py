"""The similarity graph built on the device (sda_knn_graph; Sec. 2.4, Tanimoto
kNN of Sec. 5.1) against the oracle's definition and the input generator.

Index and count work is compared bit-exactly: the CSR row pointers and
columns are equal, and so are the weights (each is the same quotient of two
integers, |x_i and x_j| / |x_i or x_j|, in FP64).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1709_04794_gb300 import sda, synth

pytestmark = pytest.mark.gpu


def _gpu(p, k, cap, thr=0.0):
    rp, col, val = sda.sda_knn_graph(torch.from_numpy(p.x_ptr).cuda(), torch.from_numpy(p.x_col).cuda(), p.d, k,
                                     cap, thr)
    return rp.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()


@pytest.mark.parametrize("k,cap,thr", [(5, None, 0.0), (8, 20, 0.0), (6, None, 0.2), (1, 7, 0.0), (32, None, 0.0)])
def test_knn_graph_matches_oracle(k, cap, thr):
    p = synth.custom_problem(1500, 700, 14, seed=23, values="counts", n_labelled=100, k=3)
    g = _gpu(p, k, p.n if cap is None else cap, thr)
    o = oracle.knn_graph(p.x_ptr, p.x_col, p.d, k, cap=cap, threshold=thr)
    for a, b in zip(g, o):
        assert np.array_equal(a, b)


def test_knn_graph_full_size_matches_generator():
    """The 200,000-row workload's graph (k = 10, candidates through features of
    at most 96 rows): the device graph equals the input generator's."""
    p = synth.make_problem("single_mixed_200k")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    rp, col, val = _gpu(p, 10, 96)
    e1.record()
    torch.cuda.synchronize()
    print("kNN graph of 200,000 rows on the device: %.1f ms" % e0.elapsed_time(e1))
    assert np.array_equal(rp, p.s_ptr) and np.array_equal(col, p.s_col) and np.array_equal(val, p.s_val)


def test_knn_graph_builds_an_operator():
    p = synth.custom_problem(800, 300, 10, seed=29, n_labelled=80, k=4)
    rp, col, val = sda.sda_knn_graph(torch.from_numpy(p.x_ptr).cuda(), torch.from_numpy(p.x_col).cuda(), p.d, 4,
                                     p.n)
    h = sda.sda_build_operator(p.x_ptr, p.x_col, p.x_val, p.d, rp, col, val, p.labels, p.alpha, float("nan"),
                               "f64")
    sda.sda_destroy_operator(h)


@pytest.mark.parametrize("k,cap,thr", [(0, 10, 0.0), (33, 10, 0.0), (4, 0, 0.0), (4, 10, 1.5)])
def test_knn_graph_rejects_bad_arguments(k, cap, thr):
    p = synth.custom_problem(100, 50, 5, seed=31, n_labelled=20, k=3)
    with pytest.raises(sda.SDAError) as e:
        _gpu(p, k, cap, thr)
    assert e.value.code == sda.SDA_ERR_INVALID_ARG


def test_knn_graph_rejects_long_rows():
    n, d = 4, 2000
    x_ptr = np.array([0, 1500, 1501, 1502, 1503], dtype=np.int64)
    x_col = np.concatenate([np.arange(1500), [0, 1, 2]]).astype(np.int32)
    with pytest.raises(sda.SDAError) as e:
        sda.sda_knn_graph(torch.from_numpy(x_ptr).cuda(), torch.from_numpy(x_col).cuda(), d, 2, n)
    assert e.value.code == sda.SDA_ERR_UNSUPPORTED
