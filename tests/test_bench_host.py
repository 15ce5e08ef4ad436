"""Host logic of bench.py (CPU only): the recorded DRAM
traffic is taken from a committed profile only while the kernel sources hash
the same as when it was captured, and per column-pass form; the algorithmic
bytes of the batched kernels follow their stated model; the oracle leg reports
the losses its shift choice came from; the chunks cover the targets once;
the sampled clock rows are summarised as the timing rules read them."""
import os

import numpy as np

import bench
from paper_1709_04794_gb300 import synth


def _profile(tmp_path, digest, lines):
    p = tmp_path / "profile.md"
    p.write_text("\n\n".join(lines + ["sources_sha256: %s" % digest]) + "\n")
    return str(p)


def test_recorded_traffic_needs_the_current_sources(tmp_path):
    lines = ["phase3a_dram_bytes_per_launch: 2878539392", "phase3a_nohead_dram_bytes_per_launch: 5200067584"]
    cur = _profile(tmp_path, bench.sources_hash(), lines)
    assert bench.recorded_traffic("phase3a", cur) == 2878539392.0
    assert bench.recorded_traffic("phase3a_nohead", cur) == 5200067584.0
    assert bench.recorded_traffic("phase1", cur) is None              # no counters for that kernel
    stale = _profile(tmp_path, "0" * 16, lines)
    assert bench.recorded_traffic("phase3a", stale) is None          # other kernel sources
    assert bench.recorded_traffic("phase3a", str(tmp_path / "missing.md")) is None


def test_committed_profile_of_the_default_workload_parses():
    path = os.path.join(bench.ROOT, "profiles", "batched_kernels_large_1000t_2m.md")
    txt = open(path).read()
    assert "phase3a_dram_bytes_per_launch:" in txt and "sources_sha256:" in txt


def test_batched_bytes_model():
    p = synth.custom_problem(3000, 2048, 30, seed=21, values="counts", n_targets=2, n_labelled=300, k=5)
    nnz, snz, n, d = int(p.x_ptr[-1]), int(p.s_ptr[-1]), p.n, p.d
    per = bench.batched_bytes(p, "f16", 100, 1600, 16)
    # rows of X: int32 index + FP16 value per entry, row pointers, P read twice, U written (FP32)
    assert per["phase1"] == nnz * 6 + (n + 1) * 8 + d * 16 * 2 * 4 + n * 16 * 4
    assert per["phase2"] == snz * 8 + (n + 1) * 8 + n * 16 * 9 + n * 4
    # recurrence form: 16 active shifts per iteration on average stream P and W (4 values each)
    assert per["phase3b"] == d * 16 * (8 + 5 * 4) + 16 * d * 4 * 4
    # the head layout moves the frequent columns' entries to 16-bit local rows
    info = {"head_cols": 64, "head_ranges": 2, "tail_nnz": nnz // 3}
    head = bench.batched_bytes(p, "f16", 100, 1600, 16, info=info)
    assert head["phase3a"] < per["phase3a"] + 2 * 2 * 64 * 16 * 8
    basis = bench.batched_bytes(p, "f16", 100, 1600, 16, basis=True, ns=24)
    assert basis["basis_once"] == 100 * d * 16 * 4 * 2 + 24 * d * 16 * 8
    assert all(v > 0 for v in basis.values())


def test_oracle_step_reports_the_losses_it_chose_from():
    """The bench's oracle leg returns the held-out loss of every shift beside
    the least-loss shift it chose, so a parity report can show how close the
    two shifts are where the mixed sweep chose another one."""
    p = synth.custom_problem(1500, 600, 12, seed=31, values="counts", n_targets=1, n_labelled=200, k=5,
                             shifts=(1e-3, 1e2, 5))
    W, tres, best, da, db, losses, tm = bench.oracle_step(p, 0, 15)
    assert W.shape == (5, p.d) and tres.shape == (5,) and losses.shape == (5,)
    assert best == int(np.argmin(losses)) and np.all(np.isfinite(losses))
    assert set(tm) == {"setup", "sweep", "checks", "adjoint"}


def test_chunk_size_keeps_chunks_in_flight_distinct():
    """The large workload's chunks: the requested size where the rank has
    enough targets for every stream, else one stream's share (the 64-target
    workload on two streams: two chunks of 32, never one chunk solved twice)."""
    assert bench.chunk_size(1000, 64, 2) == 64
    assert bench.chunk_size(64, 64, 2) == 32
    assert bench.chunk_size(125, 64, 2) == 63            # 1,000 targets over 8 ranks
    assert bench.chunk_size(5, 64, 1) == 5
    assert bench.chunk_size(1, 64, 2) == 1
    for t in (1, 7, 64, 125, 1000):
        for s in (1, 2, 3):
            c = bench.chunk_size(t, 64, s)
            chunks = -(-t // c)
            assert chunks >= min(s, t) and 1 <= c <= 64


def test_ranks_and_chunks_cover_every_target_once():
    """The large workload's 1,000 targets over 1, 2, 3 and 8 ranks: each rank's
    contiguous share split into its chunks covers every target exactly once,
    and every rank has at least as many chunks as streams in flight."""
    for world in (1, 2, 3, 8):
        seen = []
        for rank in range(world):
            begin, count = bench.shard(1000, rank, world)
            c = bench.chunk_size(count, bench.CHUNK, bench.STREAMS)
            chunks = bench.chunk_list(begin, count, c)
            assert len(chunks) >= bench.STREAMS
            seen += [t for t0, n in chunks for t in range(t0, t0 + n)]
        assert seen == list(range(1000)), world


def test_clock_rows_summarised():
    """nvidia-smi rows (csv, no header, no units) sampled during the timed
    region: the median SM clock under load, the maximum clock, and every
    throttle reason seen active; short rows and [N/A] clocks are skipped."""
    idle = ["0", "2070", "2070", "850.10", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]
    capped = ["0", "1980", "2070", "1400.00", "0x4", "Not Active", "Not Active", "Not Active", "Active"]
    hot = ["0", "1500", "2070", "1390.00", "0x48", "Active", "Active", "Not Active", "Not Active"]
    s = bench.ClockSampler.summarise([idle, idle, capped, ["0", "[N/A]"], ["garbage"]])
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s = bench.ClockSampler.summarise([idle, hot, hot])
    assert s["sm_mhz"] == 1500.0 and s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    assert bench.ClockSampler.summarise([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
