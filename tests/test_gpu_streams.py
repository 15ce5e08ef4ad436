"""Chunks of targets in flight at once, each on its own CUDA stream and host
thread (the benchmark's launch configuration): the library keeps no shared
mutable state between operators, and every cross-block reduction has a fixed
order, so two chunks solved concurrently give the same bits as the same chunks
solved one after the other (the sparse passes' schedule being the cached
autotuned one in both runs).  Each chunk: operator build with its targets'
labels, the batched mixed sweep with the FP64 residual check, the batched
adjoint gradient at one shift."""
import threading

import numpy as np
import pytest
import torch

from paper_1709_04794_gb300 import sda, synth

pytestmark = pytest.mark.gpu

NT = 16


@pytest.fixture(scope="module")
def prob():
    return synth.custom_problem(4000, 2048, 30, seed=61, values="counts", n_targets=2 * NT, n_labelled=300, k=5,
                                shifts=(1e-3, 1e2, 6))


def _chunk(p, c, stream):
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k))).cuda()
           for k in ("x_ptr", "x_col", "x_val", "s_ptr", "s_col", "s_val", "labels")}
    with torch.cuda.stream(stream):
        h = sda.sda_build_operator(dev["x_ptr"], dev["x_col"], dev["x_val"], p.d, dev["s_ptr"], dev["s_col"],
                                   dev["s_val"], dev["labels"][c * NT:(c + 1) * NT], p.alpha, float("nan"), "f16",
                                   stream)
        try:
            ns = len(p.shifts)
            w = torch.empty((NT, ns, p.d), dtype=torch.float64, device="cuda")
            o = sda.sda_default_opts()
            o.fixed_iters, o.batch_targets, o.check_residual = 40, 1, 1
            code, rep = sda.sda_solve_shifts(h, p.shifts, o, w_out=w, n_report=NT, stream=stream)
            assert code == sda.SDA_OK
            rows = np.concatenate([p.heldout[c * NT + i] for i in range(NT)]).astype(np.int64)
            off = np.concatenate([[0], np.cumsum([p.heldout[c * NT + i].size for i in range(NT)])])
            g = torch.from_numpy(np.random.default_rng(c).standard_normal(rows.size) * 1e-3).cuda()
            oa = sda.sda_default_opts()
            oa.fixed_iters = 40
            code_a, da, db, _ = sda.sda_adjoint_grad_batched(h, list(range(NT)), float("nan"),
                                                             [float(p.shifts[2])] * NT, w[:, 2].contiguous(), g,
                                                             torch.from_numpy(rows).cuda(), off, oa, stream=stream)
            assert code_a == sda.SDA_OK
            stream.synchronize()
            tres = np.array([[r["true_residual"] for r in tr] for tr in rep])
            return w.cpu().numpy(), tres, np.asarray(da), np.asarray(db)
        finally:
            sda.sda_destroy_operator(h)


def test_two_chunks_in_flight_equal_sequential(prob):
    s0 = torch.cuda.current_stream()
    _chunk(prob, 0, s0)                      # first batched run: the autotuner picks and caches the schedule
    seq = [_chunk(prob, c, s0) for c in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    res, errs = [None, None], []

    def run(c):
        try:
            res[c] = _chunk(prob, c, streams[c])
        except BaseException as e:
            errs.append(e)

    th = [threading.Thread(target=run, args=(c,)) for c in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for c in range(2):
        for a, b in zip(res[c], seq[c]):
            assert np.array_equal(a, b), c
