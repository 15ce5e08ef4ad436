"""Host logic of the multi-GPU benchmark on CPU (gloo, world size 2): the
batched workload shards its independent targets over the ranks (contiguous
shares, no exchange in the data path), and the job's time is the slowest
rank's barrier-to-barrier window; the targets solved are summed over the
ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def test_shard_covers_targets_once():
    for total in (0, 1, 5, 16, 256, 1000):
        for world in (1, 2, 3, 8):
            spans = [bench.shard(total, r, world) for r in range(world)]
            covered = [t for b, c in spans for t in range(b, b + c)]
            assert covered == list(range(total))
            sizes = [c for _, c in spans]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        begin, count = bench.shard(256, rank, world)
        t = bench.max_over_ranks(1.0 + rank, dist)        # rank 1 is the slower one
        tot = bench.sum_over_ranks(count, dist)           # targets solved by the job
        dist.barrier()
        out[rank] = (begin, count, t, tot)
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][:2] == (0, 128) and res[1][:2] == (128, 128)
    assert res[0][2] == pytest.approx(2.0) and res[1][2] == pytest.approx(2.0)
    assert res[0][3] == 256.0 and res[1][3] == 256.0
