"""Benchmark: SDA solves per second (a solve = one binary target, all its
beta shifts, converged) on the single-target 200,000 x 131,072 workload
(FP16 count values, 32 shifts 1e-5..1e3, kNN Jaccard graph k=10), plus the
achieved HBM bandwidth of the dominant kernel against the measured peak.

One step = one pass of the whole hot path over the inputs resident in HBM:
operator build (CSR->CSC, feature order, degrees, class means), shifted CG
to tol for every shift, FP64 true-residual check of every shift, and the
ratings s = X w of every shift.

  python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

N > 1 (torchrun, one process per GPU) runs independent replicas: the
single-target solve does not shard.  --impl reference times the FP64 CPU
oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "single_mixed_200k"
METRIC = "SDA solves/s (all shifts)"
UNIT = "solves/s"
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "cg_kernels_single_mixed_200k.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--compute", default=None, help="storage dtype of X (default: the workload's)")
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--max-iter", type=int, default=4000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=500,
                    help="reference arm: oracle iterations per timed step (a bounded sample of the solve)")
    ap.add_argument("--baseline-iters", type=int, default=0,
                    help="cpu_baseline of our arm: oracle iterations timed once (0: the whole solve, ~10 s on "
                         "16 cores)")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="single_mixed_200k (default); batched_256t_200k: 256 targets solved in batches of "
                         "16 that share every pass over X and S; regression_200k: CSR-SDA's regression step "
                         "(X^T X + beta I) w = X^T z on the same X; sa_200k: SA-SDA, the SDA operator with X = I_N on the "
                         "same graph and labels")
    ap.add_argument("--targets", type=int, default=0, help="batched workload: solve only the first T targets")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 9:
                for k, name in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------

KERNEL_SOURCES = ("sda_common.cuh", "sda_operator.cuh", "sda_kernels.cuh")


def sources_hash() -> str:
    """Hash of the files that define the iteration kernels (their traffic
    changes only when these do)."""
    csrc = os.path.join(ROOT, "paper_1709_04794_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(phase: str):
    """DRAM bytes per launch of the `phase` kernel from the committed ncu
    summary, if it was taken on the current kernel sources (else None)."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    txt = open(PROFILE_SUMMARY).read()
    m = re.search(r"sources_sha256:\s*([0-9a-f]+)", txt)
    t = re.search(r"%s_dram_bytes_per_launch:\s*([0-9.eE+]+)" % phase, txt)
    if not m or not t or m.group(1) != sources_hash():
        return None
    return float(t.group(1))


def algorithmic_bytes(prob, compute: str, iters: int, shift_iters: int, info: dict):
    """Algorithmic bytes per launch of each iteration kernel, averaged over one solve.

    Counted on the stored layouts with their nonzeros only (the zero padding of
    segments to whole quads, and re-reads through L2, are not algorithmic):
    phase1 (rows of X, k_rowhead):  int32 indices + values + row pointers, the
                           {r_k, p_{k-1}} pairs once each, ut written.
    phase2 (rows of S):    CSR of S (vector-type weights) + row pointers, ut
                           read once, degrees, labels, v written.
    phase3a (columns of X, k_colblk): 16-bit indices + values + the R ranges'
                           column pointers, v read once, the R ranges' partial
                           sums (pairs of the vector type) written; its stream
                           warps read r_k once and, per active shift, read and
                           write P and W.
    phase3b (stream):      the R partial sums, {r_k, p_{k-1}} and mu_l read,
                           {r_{k+1}, p_k} written."""
    n, d = prob.n, prob.d
    nnz = int(prob.x_ptr[-1])
    snz = int(prob.s_ptr[-1])
    vsz = {"f64": 8, "f32": 4, "f16": 2, "f8e4m3": 1, "pattern": 0}[compute]
    fsz = 8 if compute == "f64" else 4
    psz = 8                       # one partial sum: an FP32 pair, or an FP64 value
    mus = fsz                     # mu_l in the vector type
    R = int(info["col_ranges"])
    return {
        "phase1": nnz * (4 + vsz) + (n + 1) * 8 + 2 * d * fsz + n * fsz,
        "phase2": snz * (4 + fsz) + (n + 1) * 8 + 3 * n * fsz + n,
        "phase3a": (nnz * (2 + vsz) + R * (d + 1) * 8 + n * fsz + R * d * psz + d * fsz
                    + (shift_iters / max(iters, 1)) * d * 4 * fsz),
        "phase3b": d * (R * psz + 4 * fsz + mus),
    }


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        pk = json.load(open(path))
        return float(pk["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle as it stands
# ---------------------------------------------------------------------------

def run_reference(args, prob, rank):
    import oracle
    if rank != 0:
        return
    cores = oracle.set_threads(os.cpu_count() or 1)
    o = oracle.from_problem(prob)
    b = o.rhs_canonical()
    # iterations of the full solve (setup, untimed): the oracle's own run to tol
    full = o.shifted_cg(b, prob.shifts, tol=args.tol, max_iter=args.max_iter)
    iters_full = int(full.total_iters)
    k = max(1, min(args.cpu_iters, iters_full))
    for _ in range(args.warmup):
        o.shifted_cg(b, prob.shifts, fixed_iters=k)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.shifted_cg(b, prob.shifts, fixed_iters=k)
        times.append(time.perf_counter() - t0)
    per_solve = statistics.mean(times) * iters_full / k
    value = 1.0 / per_solve
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per_solve * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "tol": args.tol, "shifts": len(prob.shifts)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d of the %d shifted-CG iterations of the full solve per step, "
                                       "extrapolated linearly" % (k, iters_full)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def shard(total: int, rank: int, world: int):
    """Targets [begin, begin + count) of `rank` among `world` ranks: contiguous,
    sizes differing by at most one."""
    base, extra = divmod(total, world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def max_over_ranks(t_local: float, dist=None) -> float:
    """Slowest rank's time (the barrier-to-barrier window of the whole job)."""
    if dist is None:
        return t_local
    import torch
    backend = dist.get_backend()
    dev = "cuda" if backend == "nccl" else "cpu"
    t = torch.tensor([t_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def batched_bytes(prob, compute: str, batch_iters: int, shift_iters: int, ntargets: int):
    """Algorithmic bytes per launch of the batched kernels (16 targets per
    batch), averaged over the solve: X and S streamed once per launch for the
    batch, the 16 targets' vectors read / written once each, and the active
    (target, shift) pairs' P and W read and written."""
    n, d = prob.n, prob.d
    nnz = int(prob.x_ptr[-1])
    snz = int(prob.s_ptr[-1])
    vsz = {"f64": 8, "f32": 4, "f16": 2, "f8e4m3": 1, "pattern": 0}[compute]
    fsz = 8 if compute == "f64" else 4
    tb = 16
    return {
        "phase1": nnz * (4 + vsz) + (n + 1) * 8 + d * tb * 2 * fsz + n * tb * fsz,
        "phase2": snz * (4 + fsz) + (n + 1) * 8 + n * tb * (2 * fsz + 1) + n * fsz,
        "phase3a": nnz * (4 + vsz) + (d + 1) * 8 + n * tb * fsz + d * tb * 8,
        "phase3b": d * tb * (8 + 4 * fsz + fsz) + (shift_iters / max(batch_iters, 1)) * d * 4 * fsz,
    }


def run_batched(args, rank, world, local):
    """Batched sweep: all targets of the workload, one batched shifted-CG solve."""
    import torch
    from paper_1709_04794_gb300 import sda, synth
    prob = synth.make_problem(args.workload, n_targets=args.targets or None)
    compute = args.compute or prob.workload.value_dtype
    T_all = prob.labels.shape[0]
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        # targets are independent solves: each rank takes its share, no exchange
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    t_begin, T = shard(T_all, rank, world)
    stream = torch.cuda.current_stream()
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(prob, k))).cuda()
           for k in ("x_ptr", "x_col", "x_val", "s_ptr", "s_col", "s_val", "labels")}
    ns, d = len(prob.shifts), prob.d
    w = torch.empty((T, ns, d), dtype=torch.float64, device="cuda")

    def opts(profile=0, check=0, begin=t_begin, count=T):
        o = sda.sda_default_opts()
        o.tol, o.max_iter, o.check_residual, o.profile = args.tol, args.max_iter, check, profile
        o.batch_targets, o.target_begin, o.target_count = 1, begin, count
        return o

    def build():
        return sda.sda_build_operator(dev["x_ptr"], dev["x_col"], dev["x_val"], d, dev["s_ptr"], dev["s_col"],
                                      dev["s_val"], dev["labels"], prob.alpha, float("nan"), compute, stream)

    def step():
        h = build()
        try:
            code, rep = sda.sda_solve_shifts(h, prob.shifts, opts(), w_out=w, n_report=T, stream=stream)
            stats = sda.sda_get_solve_stats(h)
        finally:
            sda.sda_destroy_operator(h)
        return code, rep, stats

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = sda.sda_kernel_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        code, rep, stats = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    launches = sda.sda_kernel_launch_count() - l0
    clk = clocks.stop()
    t = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, dist)
    value = T_all * args.steps / t
    # per-kernel durations and FP64 true residuals on the first batch (untimed)
    h = build()
    try:
        w1 = torch.empty((16, ns, d), dtype=torch.float64, device="cuda")
        sda.sda_solve_shifts(h, prob.shifts, opts(profile=1, count=min(16, T)), w_out=w1, n_report=min(16, T),
                             stream=stream)
        pst = sda.sda_get_solve_stats(h)
        _, rep1 = sda.sda_solve_shifts(h, prob.shifts, opts(check=1, count=min(16, T)), w_out=w1,
                                       n_report=min(16, T), stream=stream)
    finally:
        sda.sda_destroy_operator(h)
    bi = max(1, pst["iterations"])
    per = batched_bytes(prob, compute, bi, pst["shift_iterations"], min(16, T))
    durs = {k: pst["ms"][i + 1] / bi for i, k in enumerate(("phase1", "phase2", "phase3a", "phase3b"))}
    dominant = max(durs, key=durs.get)
    peak, peak_kind = load_peaks()
    names = {"phase1": "kb_phase1 (rows of X, 16 targets)", "phase2": "kb_phase2 (rows of S, 16 targets)",
             "phase3a": "kb_phase3a (columns of X, 16 targets)", "phase3b": "kb_phase3b (vector and shift stream)"}
    achieved = per[dominant] / (durs[dominant] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": names[dominant], "peak_kind": peak_kind,
                "bytes_per_launch": per[dominant], "ms_per_launch": durs[dominant],
                "all_kernels": {names[k]: {"ms_per_launch": durs[k], "GB/s": per[k] / (durs[k] * 1e-3) / 1e9}
                                for k in durs}}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32" if compute != "f64" else "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": prob.n, "d": d, "nnz": int(prob.x_ptr[-1]), "targets": T_all,
                       "parallelism": "targets sharded over %d GPU(s), no exchange" % world,
                       "shifts": ns, "tol": args.tol, "x_storage": compute, "batch": 16,
                       "iterations": stats["iterations"], "shift_iterations": stats["shift_iterations"],
                       "status": code, "first_batch_max_true_residual":
                           max(r["true_residual"] for tr in rep1 for r in tr),
                       "l2": "no flush: one batch iteration streams > 126 MB"},
            "roofline": roofline, "cpu_baseline": None, "e2e": None, "clocks": clk, "gpu_launches": int(launches)}
    if rank == 0:
        print(json.dumps(line), flush=True)


REG_SHIFTS = np.array([1e-9, 1e-8, 1e-7, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1, 1.0, 10.0, 100.0])


def run_regression(args, rank, world, local):
    """CSR-SDA's regression step (Algorithm 5, line 5) on the X of the default
    workload: shifted CG on (X^T X + beta I) w = X^T z, z ~ U(-1, 1)^N seeded,
    the twelve beta of the paper's CG / shifted-CG comparison (Table "shifted",
    tol 1e-3); a step = build of the X^T X operator + solve + FP64 residual
    check.  The twelve single-shift CG solves are timed once after the steps
    (same tolerance) for the paper's like-for-like speed-up."""
    import torch
    from paper_1709_04794_gb300 import sda, synth
    prob = synth.make_problem(WORKLOAD)
    compute = args.compute or prob.workload.value_dtype
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    shifts = REG_SHIFTS
    n, d, ns = prob.n, prob.d, len(shifts)
    max_iter = max(args.max_iter, 20000)
    z = np.random.default_rng(1709_0005).uniform(-1.0, 1.0, n)
    rows = np.repeat(np.arange(n), np.diff(prob.x_ptr))
    b = np.bincount(prob.x_col, weights=prob.x_val * z[rows], minlength=d)      # X^T z (input)
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(prob, k))).cuda() for k in ("x_ptr", "x_col", "x_val")}
    b_dev = torch.from_numpy(b[None, :].copy()).cuda()
    w = torch.empty((1, ns, d), dtype=torch.float64, device="cuda")

    def opts(profile=0, check=1):
        o = sda.sda_default_opts()
        o.tol, o.max_iter, o.check_residual, o.profile = args.tol, max_iter, check, profile
        o.rhs_mode = sda.SDA_RHS_GIVEN
        return o

    def step(profile=0):
        h = sda.sda_build_regression(dev["x_ptr"], dev["x_col"], dev["x_val"], d, compute, stream)
        try:
            code, rep = sda.sda_solve_shifts(h, shifts, opts(profile), w_out=w, n_report=1, stream=stream,
                                             rhs=b_dev)
            stats = sda.sda_get_solve_stats(h)
            stats["info"] = sda.sda_get_operator_info(h)
        finally:
            sda.sda_destroy_operator(h)
        return code, rep, stats

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = sda.sda_kernel_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        code, rep, stats = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = sda.sda_kernel_launch_count() - l0
    clk = clocks.stop()
    t = ev0.elapsed_time(ev1) / 1e3
    # the paper's comparison: one CG solve per shift (same operator, tolerance and right-hand side)
    h = sda.sda_build_regression(dev["x_ptr"], dev["x_col"], dev["x_val"], d, compute, stream)
    w1 = torch.empty((1, 1, d), dtype=torch.float64, device="cuda")
    try:
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        cg_iters, cg_codes = [], []
        c0.record(stream)
        for beta in shifts:
            cc, _ = sda.sda_solve_shifts(h, [float(beta)], opts(check=0), w_out=w1, n_report=1, stream=stream,
                                         rhs=b_dev)
            cg_codes.append(cc)
            cg_iters.append(sda.sda_get_solve_stats(h)["iterations"])
        c1.record(stream)
        torch.cuda.synchronize()
        shifted_ms = None
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        sda.sda_solve_shifts(h, shifts, opts(check=0), w_out=w, n_report=1, stream=stream, rhs=b_dev)
        s1.record(stream)
        torch.cuda.synchronize()
        shifted_ms = s0.elapsed_time(s1)
    finally:
        sda.sda_destroy_operator(h)
    cg_ms = c0.elapsed_time(c1)
    comparison = {"cg_ms": cg_ms, "shifted_cg_ms": shifted_ms, "speedup": cg_ms / shifted_ms,
                  "cg_iterations": cg_iters, "cg_status": cg_codes,
                  "paper": "Table shifted: 43.11 s vs 6.02 s, 7.16x (ChEMBL, CPU)"}
    pcode, prep, pst = step(profile=1)
    iters = max(1, pst["iterations"])
    empty = synth.Problem(prob.workload, prob.x_ptr, prob.x_col, prob.x_val, np.zeros(n + 1, np.int64),
                          np.zeros(0, np.int32), np.zeros(0), prob.labels, prob.truth, prob.heldout,
                          shifts, 0.0)
    per = algorithmic_bytes(empty, compute, pst["iterations"], pst["shift_iterations"], pst["info"])
    durs = {k: pst["ms"][i + 1] / iters for i, k in enumerate(("phase1", "phase2", "phase3a", "phase3b"))}
    dominant = max(durs, key=durs.get)
    peak, peak_kind = load_peaks()
    names = {"phase1": "k_rowhead (rows of X)", "phase2": "k_rowpass<EpiP2> (identity rows)",
             "phase3a": "k_colblk (columns of X, shift stream)", "phase3b": "k_cg_phase3b (vector stream)"}
    achieved = per[dominant] / (durs[dominant] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": names[dominant], "peak_kind": peak_kind,
                "bytes_per_launch": per[dominant], "ms_per_launch": durs[dominant],
                "all_kernels": {names[k]: {"ms_per_launch": durs[k], "GB/s": per[k] / (durs[k] * 1e-3) / 1e9}
                                for k in durs}}
    line = {"metric": "regression solves/s (all shifts)", "value": args.steps / t, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if compute != "f64" else "f64", "data": "synthetic",
            "config": {"workload": "regression_200k", "n": n, "d": d, "nnz": int(prob.x_ptr[-1]), "shifts": ns,
                       "tol": args.tol, "x_storage": compute, "iterations": stats["iterations"],
                       "shift_iterations": stats["shift_iterations"], "status": code,
                       "max_true_residual": max(r["true_residual"] for r in rep[0]),
                       "shift_values": "Table shifted, first row", "cg_vs_shifted_cg": comparison},
            "roofline": roofline, "cpu_baseline": None, "e2e": None, "clocks": clk, "gpu_launches": int(launches)}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_sa(args, rank, world, local):
    """SA-SDA (Algorithm 6) on the graph and labels of the default workload: the
    SDA operator with X = I_N (N = 200,000 unknowns), its 32 shifts, tol 1e-3;
    a step = build + solve + FP64 residual check; the rating is the solution."""
    import dataclasses
    import torch
    from paper_1709_04794_gb300 import sda, synth
    prob = synth.make_problem(WORKLOAD)
    compute = args.compute or prob.workload.value_dtype
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    n, ns = prob.n, len(prob.shifts)
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(prob, k))).cuda()
           for k in ("s_ptr", "s_col", "s_val", "labels")}
    z = torch.empty((1, ns, n), dtype=torch.float64, device="cuda")

    def opts(profile=0):
        o = sda.sda_default_opts()
        o.tol, o.max_iter, o.check_residual, o.profile = args.tol, args.max_iter, 1, profile
        return o

    def step(profile=0):
        h = sda.sda_build_sa(dev["s_ptr"], dev["s_col"], dev["s_val"], dev["labels"], prob.alpha, float("nan"),
                             compute, stream)
        try:
            code, rep = sda.sda_solve_shifts(h, prob.shifts, opts(profile), w_out=z, n_report=1, stream=stream)
            stats = sda.sda_get_solve_stats(h)
            stats["info"] = sda.sda_get_operator_info(h)
        finally:
            sda.sda_destroy_operator(h)
        return code, rep, stats

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = sda.sda_kernel_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        code, rep, stats = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = sda.sda_kernel_launch_count() - l0
    clk = clocks.stop()
    t = ev0.elapsed_time(ev1) / 1e3
    pcode, prep, pst = step(profile=1)
    iters = max(1, pst["iterations"])
    ident = synth.Problem(dataclasses.replace(prob.workload, d=n), np.arange(n + 1, dtype=np.int64),
                          np.arange(n, dtype=np.int32), np.ones(n), prob.s_ptr, prob.s_col, prob.s_val,
                          prob.labels, prob.truth, prob.heldout, prob.shifts, prob.alpha)
    per = algorithmic_bytes(ident, compute, pst["iterations"], pst["shift_iterations"], pst["info"])
    durs = {k: pst["ms"][i + 1] / iters for i, k in enumerate(("phase1", "phase2", "phase3a", "phase3b"))}
    dominant = max(durs, key=durs.get)
    peak, peak_kind = load_peaks()
    names = {"phase1": "k_rowhead (rows of I)", "phase2": "k_rowpass<EpiP2> (rows of S)",
             "phase3a": "k_colblk (columns of I, shift stream)", "phase3b": "k_cg_phase3b (vector stream)"}
    achieved = per[dominant] / (durs[dominant] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": names[dominant], "peak_kind": peak_kind,
                "bytes_per_launch": per[dominant], "ms_per_launch": durs[dominant],
                "all_kernels": {names[k]: {"ms_per_launch": durs[k], "GB/s": per[k] / (durs[k] * 1e-3) / 1e9}
                                for k in durs}}
    line = {"metric": "SA-SDA solves/s (all shifts)", "value": args.steps / t, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if compute != "f64" else "f64", "data": "synthetic",
            "config": {"workload": "sa_200k", "n": n, "graph_nnz": int(prob.s_ptr[-1]), "shifts": ns,
                       "tol": args.tol, "alpha": prob.alpha, "iterations": stats["iterations"],
                       "shift_iterations": stats["shift_iterations"], "status": code,
                       "max_true_residual": max(r["true_residual"] for r in rep[0])},
            "roofline": roofline, "cpu_baseline": None, "e2e": None, "clocks": clk, "gpu_launches": int(launches)}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "sa_200k" and args.impl == "ours":
        run_sa(args, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
               int(os.environ.get("LOCAL_RANK", "0")))
        return
    if args.workload == "regression_200k" and args.impl == "ours":
        run_regression(args, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
                       int(os.environ.get("LOCAL_RANK", "0")))
        return
    if args.workload != WORKLOAD and args.impl == "ours":
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        local = int(os.environ.get("LOCAL_RANK", "0"))
        run_batched(args, rank, world, local)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_1709_04794_gb300 import synth
    prob = synth.make_problem(WORKLOAD)
    compute = args.compute or prob.workload.value_dtype
    if args.impl == "reference":
        run_reference(args, prob, rank)
        return

    import torch
    from paper_1709_04794_gb300 import sda
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.current_stream()
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(prob, k))).cuda()
           for k in ("x_ptr", "x_col", "x_val", "s_ptr", "s_col", "s_val", "labels")}
    ns, d, n = len(prob.shifts), prob.d, prob.n
    w = torch.empty((1, ns, d), dtype=torch.float64, device="cuda")
    scores = torch.empty((ns, n), dtype=torch.float64, device="cuda")

    def opts(profile=0, out_dev=1):
        o = sda.sda_default_opts()
        o.tol, o.max_iter, o.check_residual, o.profile = args.tol, args.max_iter, 1, profile
        o.out_on_device = out_dev
        return o

    def step(profile=0):
        h = sda.sda_build_operator(dev["x_ptr"], dev["x_col"], dev["x_val"], d, dev["s_ptr"], dev["s_col"],
                                   dev["s_val"], dev["labels"], prob.alpha, float("nan"), compute, stream)
        try:
            code, rep = sda.sda_solve_shifts(h, prob.shifts, opts(profile), w_out=w, n_report=1, stream=stream)
            sda.sda_project(h, w[0], ns, scores, 0, 0, stream)
            stats = sda.sda_get_solve_stats(h)
            stats["info"] = sda.sda_get_operator_info(h)
        finally:
            sda.sda_destroy_operator(h)
        return code, rep, stats

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = sda.sda_kernel_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    ev0.record(stream)
    reports = []
    for _ in range(args.steps):
        reports.append(step())
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = sda.sda_kernel_launch_count() - l0
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    t_local = ms / 1e3
    if dist is not None:
        t = torch.tensor([t_local], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    else:
        t_max = t_local
    value = world * args.steps / t_max
    code, rep, stats = reports[-1]

    # per-kernel durations: one profiled solve (events around every phase kernel)
    pcode, prep, pstats = step(profile=1)
    pinfo = pstats["info"]
    iters = max(1, pstats["iterations"])
    per_launch = algorithmic_bytes(prob, compute, pstats["iterations"], pstats["shift_iterations"], pinfo)
    durs = {k: pstats["ms"][i + 1] / iters for i, k in enumerate(("phase1", "phase2", "phase3a", "phase3b"))}
    dominant = max(durs, key=durs.get)
    peak, peak_kind = load_peaks()
    achieved = per_launch[dominant] / (durs[dominant] * 1e-3) / 1e9
    kernel_names = {"phase1": "k_rowhead (rows of X)", "phase2": "k_rowpass<EpiP2> (rows of S)",
                    "phase3a": "k_colblk (columns of X, shift stream)", "phase3b": "k_cg_phase3b (vector stream)"}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": recorded_traffic(dominant),
                "kernel": kernel_names[dominant], "peak_kind": peak_kind,
                "bytes_per_launch": per_launch[dominant], "ms_per_launch": durs[dominant],
                "all_kernels": {kernel_names[k]: {"ms_per_launch": durs[k], "GB/s": per_launch[k] / (durs[k] * 1e-3) / 1e9}
                                for k in durs}}

    # end to end through the C ABI with host buffers: the inputs sit in pinned
    # host memory (filled before the timed region), the solutions come back to
    # a pinned host array
    e2e = None
    if not args.no_e2e:
        host = {k: torch.from_numpy(np.ascontiguousarray(getattr(prob, k))).pin_memory() for k in
                ("x_ptr", "x_col", "x_val", "s_ptr", "s_col", "s_val", "labels")}
        w_host = torch.empty((1, ns, d), dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        d2h = w_host.numel() * w_host.element_size() + ns * 24
        e_steps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            h = sda.sda_build_operator(host["x_ptr"], host["x_col"], host["x_val"], d, host["s_ptr"], host["s_col"],
                                       host["s_val"], host["labels"], prob.alpha, float("nan"), compute, stream)
            try:
                sda.sda_solve_shifts(h, prob.shifts, opts(0, 0), w_out=w_host, n_report=1, stream=stream)
            finally:
                sda.sda_destroy_operator(h)
        el = time.perf_counter() - t0
        e2e = {"value": world * e_steps / el, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": e_steps,
               "step": "H2D of X, S and labels from pinned host memory, operator build, solve with the FP64 "
                       "residual check, D2H of w to pinned host memory (no projection)"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle
        cores = oracle.set_threads(os.cpu_count() or 1)
        o = oracle.from_problem(prob)
        b = o.rhs_canonical()
        k = min(args.baseline_iters, iters) if args.baseline_iters > 0 else iters
        o.shifted_cg(b, prob.shifts, fixed_iters=3)
        t0 = time.perf_counter()
        o.shifted_cg(b, prob.shifts, fixed_iters=k)
        el = time.perf_counter() - t0
        cpu = {"value": 1.0 / (el * stats["iterations"] / k), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": ("one whole solve: %d shifted-CG iterations of the FP64 oracle (the iterations of "
                          "the GPU solve)" % k) if k == stats["iterations"] else
                         ("%d of the %d shifted-CG iterations of one solve (FP64 oracle), extrapolated linearly"
                          % (k, stats["iterations"]))}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if compute != "f64" else "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": n, "d": d, "nnz": int(prob.x_ptr[-1]),
                           "graph_nnz": int(prob.s_ptr[-1]), "x_storage": compute, "shifts": ns, "tol": args.tol,
                           "alpha": prob.alpha, "iterations": stats["iterations"],
                           "shift_iterations": stats["shift_iterations"],
                           "max_true_residual": max(r["true_residual"] for r in rep[0]),
                           "status": code, "parallelism": "replicas" if world > 1 else "single",
                           "l2": "no flush: one iteration streams ~%d MB (> 126 MB L2)"
                                 % int(sum(per_launch.values()) / 1e6)},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": int(launches)}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
