"""Throughput of the trajectory-kNN rarity path on GB300.

One step = one full forward pass (centring, operand preparation with FP64 day
norms, fused Gram/window/top-k kernel, merge and scores) over the 75-year
European workload: N = 27,394 daily fields on a 46 x 81 grid (D = 3,726),
L = 5, k = 20, exclusion 4, SLP-like synthetic data.

Metric: trajectory pairs per second, pairs = M^2 ordered trajectory pairs
resolved per step (M = N - L + 1). The headline value is the split-BF16
tensor-core path; the plain FP32 CUDA-core path is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own independent series (weak
scaling); value = all pairs resolved / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("trajectory pairs/s, split-BF16 vs FP32 path (75y×3726pt, L=5, k=20); "
          "% roofline")
WORKLOAD = "euro_75y_46x81"
L2_BYTES = 129e6
PROFILE_DIR = os.path.join(ROOT, "profiles")


# --------------------------------------------------------------------- helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value: float, ws: int, device=None) -> float:
    """Max over ranks (identity for a single process)."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(pairs_per_rank: float, ms_per_step_max: float, ws: int) -> float:
    """Whole-job throughput: all ranks' pairs over the slowest rank's step time."""
    return pairs_per_rank * ws / (ms_per_step_max * 1e-3)


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.out = None

    def start(self):
        try:
            self.out = open(os.devnull, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            txt, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            txt, _ = self.proc.communicate()
        return parse_clocks(txt)


def parse_clocks(txt: str):
    rows = [r for r in csv.reader(io.StringIO(txt)) if len(r) >= 9]
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
    smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = set()
    for r in rows:
        for n, v in zip(names, r[5:9]):
            if v.strip().lower() == "active":
                reasons.add(n)
    load = [v for v in sm if smax and v > 0.5 * max(smax)] or sm
    return {"sm_mhz": statistics.median(load) if load else None,
            "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
            "samples": len(rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "fallback"


def kernel_traffic():
    """DRAM bytes per step of the fused kernel (band + main launch) from the committed
    ncu summary, if it was taken on the current kernel source (digest match)."""
    import hashlib
    import re
    p = os.path.join(PROFILE_DIR, "fused_tc_kernel__euro_75y_46x81__dram.md")
    try:
        with open(p) as f:
            txt = f.read()
        with open(os.path.join(ROOT, "paper_2603_02059_gb300", "csrc", "kernel_tc.cu"), "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    m_b = re.search(r"^traffic_bytes_per_step:\s*(\d+)", txt, re.M)
    m_d = re.search(r"^source_digest:\s*([0-9a-f]+)", txt, re.M)
    if not m_b or not m_d or m_d.group(1) != digest:
        return None
    return float(m_b.group(1))


# --------------------------------------------------------------- our arm

def run_ours(args, ws, rank, local):
    import torch

    import paper_2603_02059_gb300 as tk
    from synth import config_inputs

    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)

    # weak scaling: every rank its own series; --split: one series shared by all ranks
    X, meta, cfg = config_inputs(args.workload, seed_offset=0 if args.split else rank)
    N, D = X.shape
    L, k, e = cfg["L"], cfg["k"], cfg["exclusion"]
    M = N - L + 1
    pairs = float(M) * M
    Xd = torch.from_numpy(X).to(device)
    out = (torch.empty((M, k), dtype=torch.int32, device=device),
           torch.empty((M, k), dtype=torch.float32, device=device),
           torch.empty((M,), dtype=torch.float32, device=device))
    h = tk.get_handle(local)
    stream = torch.cuda.current_stream(device)

    def step(prec):
        if args.split and prec != "fp32":
            if ws > 1:
                tk.knn_scores_split(Xd, L, k, e, precision=prec, handle=h)
            else:
                ip, dp = tk.knn_partial(Xd, L, k, e, 0, 1, precision=prec, handle=h)
                tk.merge_partials(ip[None], dp[None], handle=h)
        else:
            tk.knn_scores(Xd, L, k, e, precision=prec, handle=h, out=out)

    def timed(prec, steps, warmup, sample_clocks=False):
        for _ in range(warmup):
            step(prec)
        torch.cuda.synchronize(device)
        h.profile_read()
        h.set_option("profile", 1)
        n0 = h.launch_count()
        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        barrier(ws)
        torch.cuda.synchronize(device)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step(prec)
        e1.record(stream)
        torch.cuda.synchronize(device)
        barrier(ws)
        clocks = sampler.stop() if sampler else None
        launches = h.launch_count() - n0
        kms = h.profile_read()
        h.set_option("profile", 0)
        if h.sync_status() != 0:
            raise RuntimeError("device-side failure during the timed region")
        ms = e0.elapsed_time(e1) / steps
        return reduce_max(ms, ws, device), kms, launches, clocks

    # headline: split-BF16 tensor-core path
    head = args.headline
    ms_split, kms_split, launches, clocks = timed(head, args.steps, args.warmup, True)
    # split: the ranks share one series' pairs; otherwise every rank resolves its own
    value = aggregate(pairs / ws if args.split else pairs, ms_split, ws)
    # plain FP32 CUDA-core path on the same input
    fp32_steps = max(1, min(args.steps, args.fp32_steps))
    if args.skip_fp32:
        ms_fp32, kms_fp32 = None, []
    else:
        ms_fp32, kms_fp32, _, _ = timed("fp32", fp32_steps, 1)

    # roofline of the dominant kernel (fused Gram/window/top-k launches): executed
    # tensor work = N(N+1)/2 day pairs x 2D flops x 3 products (split-BF16; 1 for BF16),
    # algorithmic work = the method's own N(N+1)/2 x 2D (one product per pair)
    peaks, peak_src = measured_peaks()
    products = 3 if head == "split_bf16" else 1
    algo_flops = N * (N + 1) / 2 * 2 * D / (ws if args.split else 1)  # this rank's share
    flops = algo_flops * products
    kavg = statistics.mean(kms_split) * 1e-3 if kms_split else None
    achieved = flops / kavg / 1e12 if kavg else None
    # the burst peak applies to a kernel timed in a region shorter than a second; the
    # sustained one (a seconds-long loop under the power cap) to a longer region
    region_s = ms_split * args.steps * 1e-3
    peak_key = "bf16_tflops" if region_s < 1.0 else "bf16_tflops_sustained"
    peak = float(peaks[peak_key])
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": kernel_traffic() if args.workload == WORKLOAD else None,
                "peak_source": f"{peak_src} {peak_key} (timed region {region_s:.2f} s)",
                "work": (f"executed: N(N+1)/2 day pairs x 2D flops x {products} "
                         f"BF16 product(s) = {flops:.4g} flop per step"),
                "achieved_algorithmic": (algo_flops / kavg / 1e12) if kavg else None,
                "frac_algorithmic": (algo_flops / kavg / 1e12 / peak) if kavg else None,
                "frac_other_peak": ((achieved / float(peaks["bf16_tflops_sustained"
                                     if peak_key == "bf16_tflops" else "bf16_tflops"]))
                                    if achieved else None),
                "kernel": "fused Gram/window/top-k (tcgen05), band pre-pass + main pass",
                "kernel_ms": statistics.mean(kms_split) if kms_split else None,
                "share_of_step": (statistics.mean(kms_split) / ms_split) if kms_split else None}

    # end to end through the public host-buffer API: pinned X in, results out
    e2e = None
    if not args.skip_e2e and not args.split:  # (the host-buffer call is single-process)
        e2e = run_e2e(tk, h, X, L, k, e, head, args.steps, ws, device)


    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_split, "higher_is_better": True,
        "scaling": "strong" if args.split else "weak", "vs_baseline": None,
        "dtype": {"split_bf16": "bf16", "bf16": "bf16", "fp32": "f32"}[head],
        "data": ("synthetic (seeded SLP-like anomalies; one series split across the ranks)"
                 if args.split else
                 "synthetic (seeded SLP-like anomalies; one independent series per rank)"),
        "config": {"workload": (f"{args.workload}: N={N} days, D={D} ({meta.h}x{meta.w}), "
                                f"L={L}, k={k}, exclusion={e}, M={M}"),
                   "pairs_per_step": pairs,
                   "precision": {"split_bf16": "split-BF16 (3 BF16 products, FP32 accumulate; "
                                               "FP64 norms)",
                                 "bf16": "BF16 (1 product, FP32 accumulate; FP64 norms)",
                                 "fp32": "FP32 CUDA cores; FP64 norms"}[head],
                   "l2": l2_note(N, D),
                   "parallelism": (f"one series, upper-triangle strips split over {ws} ranks, "
                                   f"candidate lists all-gathered once" if args.split else
                                   f"independent series per rank x{ws}")},
        "fp32_path": None if ms_fp32 is None else {
            "value": aggregate(pairs, ms_fp32, ws), "ms_per_step": ms_fp32,
            "kernel_ms": statistics.mean(kms_fp32) if kms_fp32 else None, "steps": fp32_steps,
            "roofline": fp32_roofline(N, D, kms_fp32, peaks)},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(X, L, k, e, args.cpu_rows)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line


def l2_note(N, D):
    """How the timed steps avoid running from a warm L2 (129 MB)."""
    xb = N * D * 4
    ob = N * ((D + 62) // 63) * 64 * 2 * 2
    if xb > L2_BYTES and ob > L2_BYTES:
        return (f"inputs larger than L2 (X is {xb / 1e6:.0f} MB; operand copies "
                f"{ob / 1e6:.0f} MB), no flush needed")
    return (f"X ({xb / 1e6:.1f} MB) and operand copies ({ob / 1e6:.1f} MB) fit in L2: "
            f"L2 not flushed between steps (a small-case line, not the headline)")


def fp32_roofline(N, D, kms, peaks):
    """FP32 CUDA-core path: both triangles of the Gram (N^2 x 2D flops) against the
    FP32 FMA peak of 152 SMs at the maximum SM clock."""
    if not kms:
        return None
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = fp32_alu_peak_tflops(sms, float(peaks.get("sm_max_mhz", 2070.0)))
    ach = float(N) * N * 2 * D / (statistics.mean(kms) * 1e-3) / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x sm_max_mhz"}


def run_e2e(tk, h, X, L, k, e, prec, steps, ws, device):
    """Same metric through the host-buffer entry point: every step copies X in from
    pinned memory, computes, copies the neighbour lists and scores out."""
    import torch
    M = X.shape[0] - L + 1
    pairs = float(M) * M
    Xh = torch.from_numpy(X).pin_memory()
    outh = (torch.empty((M, k), dtype=torch.int32).pin_memory(),
            torch.empty((M, k), dtype=torch.float32).pin_memory(),
            torch.empty((M,), dtype=torch.float32).pin_memory())
    for _ in range(2):
        tk.knn_scores_host(Xh, L, k, e, precision=prec, handle=h, out=outh)
    barrier(ws)
    n = max(1, steps)
    calls = []
    t0 = time.perf_counter()
    for _ in range(n):
        t1 = time.perf_counter()
        tk.knn_scores_host(Xh, L, k, e, precision=prec, handle=h, out=outh)
        calls.append((time.perf_counter() - t1) * 1e3)
    ms = reduce_max((time.perf_counter() - t0) * 1e3 / n, ws, device)
    return {"value": aggregate(pairs, ms, ws), "unit": "pairs/s", "ms_per_step": ms,
            "ms_per_call_median": statistics.median(calls), "ms_per_call_min": min(calls),
            "h2d_bytes_per_step": X.nbytes,
            "d2h_bytes_per_step": sum(t.numel() * t.element_size() for t in outh),
            "api": "traknn_knn_scores_host (pinned host buffers)"}


def cpu_baseline(X, L, k, e, nrows):
    """The FP64 oracle, as it stands, on a bounded sample of rows of the same workload."""
    import oracle
    M = X.shape[0] - L + 1
    rows = np.linspace(0, M - 1, nrows).astype(np.int64)
    t0 = time.perf_counter()
    oracle.knn_rows(X, L, k, e, rows)
    el = time.perf_counter() - t0
    # the small workload in full (all M^2 pairs), for reference
    from synth import config_inputs
    Xs, _, cs = config_inputs("small_5y_16x32")
    Ms = Xs.shape[0] - cs["L"] + 1
    t1 = time.perf_counter()
    oracle.knn_scores(Xs, cs["L"], cs["k"], cs["exclusion"])
    els = time.perf_counter() - t1
    return {"value": nrows * M / el, "unit": "pairs/s", "cores": oracle.num_threads(),
            "kind": "oracle", "seconds": el,
            "sample": f"{nrows} evenly spaced trajectory rows x all M={M} candidates "
                      f"(FP64 direct differences, full sort)",
            "small_full": {"workload": "small_5y_16x32 (N=1826, D=512, L=3, k=10), all pairs",
                           "seconds": els, "pairs_per_s": float(Ms) * Ms / els}}


# ------------------------------------------------------------ extra workloads

FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM (4 partitions x 32)


def fp32_alu_peak_tflops(sm_count: int, sm_mhz: float) -> float:
    """FP32 FMA peak from unit counts and clock: SMs x lanes x 2 flops x clock."""
    return sm_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def _events_ms(fn, steps, warmup, stream=None):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def suite_precision(args):
    """0.25-degree grid (D = 58,101), L in {3, 5, 7, 10}, k = 20: split-BF16 throughput
    per L (the cost of the diagonal window must not grow with L) and the FP32 path
    at L = 5."""
    import torch

    import paper_2603_02059_gb300 as tk
    from synth import config_inputs
    X, meta, cfg = config_inputs("euro_75y_181x321")
    N, D = X.shape
    Xd = torch.from_numpy(X).cuda()
    del X
    h = tk.get_handle()
    peaks, src = measured_peaks()
    out = []
    for L in (3, 5, 7, 10):
        k, e = cfg["k"], L - 1
        M = N - L + 1
        h.profile_read()
        h.set_option("profile", 1)
        ms = _events_ms(lambda: tk.knn_scores(Xd, L, k, e, handle=h), args.steps, 3)
        kms = h.profile_read()[3:]
        h.set_option("profile", 0)
        kavg = statistics.mean(kms) if kms else None
        flops = N * (N + 1) / 2 * 3 * 2 * D
        ach = flops / (kavg * 1e-3) / 1e12 if kavg else None
        out.append({"L": L, "k": k, "exclusion": e, "ms_per_step": ms,
                    "pairs_per_s": float(M) * M / (ms * 1e-3), "kernel_ms": kavg,
                    "tensor_tflops": ach,
                    "frac_sustained": ach / peaks["bf16_tflops_sustained"] if ach else None,
                    "frac_burst": ach / peaks["bf16_tflops"] if ach else None})
    # all four trajectory lengths from one Gram sweep
    settings = [(r["L"], r["k"], r["exclusion"]) for r in out]
    ms_multi = _events_ms(lambda: tk.knn_scores_multi(Xd, settings, handle=h), args.steps, 3)
    pairs_all = sum(float(N - r["L"] + 1) ** 2 for r in out)
    multi = {"settings": settings, "ms_per_step": ms_multi,
             "pairs_per_s": pairs_all / (ms_multi * 1e-3),
             "sum_of_single_ms": sum(r["ms_per_step"] for r in out)}
    L, k = 5, cfg["k"]
    M = N - L + 1
    ms32 = _events_ms(lambda: tk.knn_scores(Xd, L, k, L - 1, precision="fp32", handle=h), 1, 1)
    if h.sync_status() != 0:
        raise RuntimeError("device-side failure")
    return {"suite": "precision_sweep", "workload": f"euro_75y_181x321: N={N}, D={D}",
            "split_bf16": out, "multi_L_one_sweep": multi,
            "fp32_L5": {"ms_per_step": ms32, "pairs_per_s": float(M) * M / (ms32 * 1e-3)},
            "peak_source": src}


def batched_shapes(n_series=64, seed=20260305):
    """64 series of uneven length N ~ U[3650, 27394], L ~ U{2..10}, k in {5, 10, 20},
    exclusion L - 1, all on the 46 x 81 grid."""
    rng = np.random.default_rng(seed)
    shapes = []
    for _ in range(n_series):
        N = int(rng.integers(3650, 27395))
        L = int(rng.integers(2, 11))
        k = int(rng.choice([5, 10, 20]))
        shapes.append((N, L, k, L - 1))
    return shapes


def suite_batched(args):
    """64 uneven series in one batched call (persistent launches replayed from a CUDA
    graph, tiles per unit autotuned) against 64 sequential single-series calls."""
    import torch

    import paper_2603_02059_gb300 as tk
    from synth import make_slp_like
    shapes = batched_shapes()
    Xs = []
    for b, (N, L, k, e) in enumerate(shapes):
        X, _ = make_slp_like(N, 46, 81, seed=20260400 + b)
        Xs.append(torch.from_numpy(X).cuda())
    h = tk.get_handle()
    pairs = float(sum((N - L + 1) ** 2 for N, L, k, e in shapes))
    outs = [(torch.empty((N - L + 1, k), dtype=torch.int32, device="cuda"),
             torch.empty((N - L + 1, k), dtype=torch.float32, device="cuda"),
             torch.empty((N - L + 1,), dtype=torch.float32, device="cuda"))
            for N, L, k, e in shapes]
    series = [(X, L, k, e) for X, (N, L, k, e) in zip(Xs, shapes)]

    def seq():
        for (X, L, k, e), o in zip(series, outs):
            tk.knn_scores(X, L, k, e, handle=h, out=o)

    def bat():
        tk.knn_scores_batched(series, handle=h, outs=outs, autotune=True)

    ms_seq = _events_ms(seq, args.steps, 3)
    ms_bat = _events_ms(bat, args.steps, 3)
    tiles, group = h.work_shape()
    # the same batched call with the default work-unit shape (no autotuning)
    h.set_option("autotune", 0)
    ms_def = _events_ms(lambda: tk.knn_scores_batched(series, handle=h, outs=outs),
                        args.steps, 3)
    if h.sync_status() != 0:
        raise RuntimeError("device-side failure")
    return {"suite": "batched", "series": len(shapes), "D": 46 * 81,
            "total_days": sum(s[0] for s in shapes), "pairs_per_step": pairs,
            "batched": {"ms_per_step": ms_bat, "pairs_per_s": pairs / (ms_bat * 1e-3)},
            "sequential": {"ms_per_step": ms_seq, "pairs_per_s": pairs / (ms_seq * 1e-3)},
            "speedup": ms_seq / ms_bat,
            "autotuned_shape": {"tiles_per_unit": tiles, "group_strips": group},
            "default_shape_ms_per_step": ms_def, "autotune_speedup": ms_def / ms_bat}


def suite_adjoint(args):
    """30-year workload (N = 10,957, D = 3,726, L = 5, k = 10): forward pass and the
    adjoint of the summed score. The adjoint's floor is its HBM bytes (read X, idx, g;
    write dX), the fraction reported; its partner-row gather runs from L2."""
    import torch

    import paper_2603_02059_gb300 as tk
    from synth import config_inputs
    X, meta, cfg = config_inputs("euro_30y_46x81")
    N, D = X.shape
    L, k, e = cfg["L"], cfg["k"], cfg["exclusion"]
    M = N - L + 1
    Xd = torch.from_numpy(X).cuda()
    h = tk.get_handle()
    idx, dist, score = tk.knn_scores(Xd, L, k, e, handle=h)
    g = torch.ones(M, device="cuda")
    ms_fwd = _events_ms(lambda: tk.knn_scores(Xd, L, k, e, handle=h, out=(idx, dist, score)),
                        args.steps, 3)
    ms_bwd = _events_ms(lambda: tk.score_backward(Xd, L, k, idx, g, handle=h), args.steps, 3)
    if h.sync_status() != 0:
        raise RuntimeError("device-side failure")
    peaks, src = measured_peaks()
    algo = 2 * N * D * 4 + M * k * 4 + M * 4
    gbs = algo / (ms_bwd * 1e-3) / 1e9
    return {"suite": "adjoint", "workload": f"euro_30y_46x81: N={N}, D={D}, L={L}, k={k}",
            "forward_ms": ms_fwd, "forward_pairs_per_s": float(M) * M / (ms_fwd * 1e-3),
            "backward_ms": ms_bwd, "backward_algorithmic_bytes": algo,
            "backward_gbs": gbs, "hbm_peak_gbs": peaks["hbm_gbs"],
            "frac": gbs / peaks["hbm_gbs"], "peak_source": src}


def suite_ext(args):
    """75-year workload: the forward pass with cosine-of-latitude grid-point weights
    against the unweighted one, and the statistics kernel (scores for every k' <= k and
    the local intrinsic dimension) on its neighbour lists (HBM-bound: reads M k floats,
    writes M k + M floats)."""
    import torch

    import paper_2603_02059_gb300 as tk
    from synth import config_inputs
    X, meta, cfg = config_inputs(WORKLOAD)
    N, D = X.shape
    L, k, e = cfg["L"], cfg["k"], cfg["exclusion"]
    M = N - L + 1
    Xd = torch.from_numpy(X).cuda()
    h = tk.get_handle()
    out = (torch.empty((M, k), dtype=torch.int32, device="cuda"),
           torch.empty((M, k), dtype=torch.float32, device="cuda"),
           torch.empty((M,), dtype=torch.float32, device="cuda"))
    ms_plain = _events_ms(lambda: tk.knn_scores(Xd, L, k, e, handle=h, out=out), args.steps, 3)
    lat = np.deg2rad(np.linspace(72.0, 27.0, 46))
    w = torch.from_numpy(np.repeat(np.cos(lat), 81).astype(np.float32)).cuda()
    h.set_grid_weights(w)
    ms_w = _events_ms(lambda: tk.knn_scores(Xd, L, k, e, handle=h, out=out), args.steps, 3)
    h.set_grid_weights(None)
    dist = out[1]
    ms_stats = _events_ms(lambda: tk.knn_stats(dist, k_id=k, handle=h), 20, 3)
    if h.sync_status() != 0:
        raise RuntimeError("device-side failure")
    peaks, src = measured_peaks()
    nbytes = M * k * 4 * 2 + M * 4
    gbs = nbytes / (ms_stats * 1e-3) / 1e9
    # trajectory lengths 3, 5, 7, 10 from one Gram sweep on this workload
    settings = [(Lx, k, Lx - 1) for Lx in (3, 5, 7, 10)]
    ms_single = sum(_events_ms(lambda Lx=Lx: tk.knn_scores(Xd, Lx, k, Lx - 1, handle=h),
                               args.steps, 3) for Lx, _, _ in settings)
    ms_multi = _events_ms(lambda: tk.knn_scores_multi(Xd, settings, handle=h), args.steps, 3)
    multi = {"settings": settings, "ms_per_step": ms_multi, "sum_of_single_ms": ms_single}
    # time against k (the paper notes k has little influence on the cost) and N
    k_sweep = {}
    for kx in (5, 10, 20, 40, 64):
        k_sweep[kx] = _events_ms(lambda kx=kx: tk.knn_scores(Xd, L, kx, e, handle=h),
                                 args.steps, 3)
    n_sweep = {}
    for nx in (6849, 13697, 20546, N):  # about 19, 37.5, 56 and 75 years
        Xn = Xd[:nx]
        ms = _events_ms(lambda Xn=Xn: tk.knn_scores(Xn, L, k, e, handle=h), args.steps, 3)
        mx = nx - L + 1
        n_sweep[nx] = {"ms_per_step": ms, "pairs_per_s": float(mx) * mx / (ms * 1e-3)}
    # small-D form: 75 years of 32-value fields (a stand-in for PCA-reduced data)
    from synth import make_slp_like
    Xs, _ = make_slp_like(N, 4, 8, seed=20260310, annual_amp=5.0)
    Xsd = torch.from_numpy(Xs).cuda()
    small = {}
    for prec in ("split_bf16", "fp32"):
        ms = _events_ms(lambda: tk.knn_scores(Xsd, L, k, e, precision=prec, handle=h),
                        args.steps if prec == "split_bf16" else 2, 2)
        small[prec] = {"ms_per_step": ms, "pairs_per_s": float(M) * M / (ms * 1e-3)}
    if h.sync_status() != 0:
        raise RuntimeError("device-side failure")
    return {"suite": "ext", "workload": f"{WORKLOAD}: N={N}, D={D}, L={L}, k={k}",
            "forward_ms": ms_plain, "forward_weighted_ms": ms_w,
            "stats_ms": ms_stats, "stats_bytes": nbytes, "stats_gbs": gbs,
            "stats_frac_hbm": gbs / peaks["hbm_gbs"], "peak_source": src,
            "multi_L_one_sweep": multi, "ms_vs_k": k_sweep, "ms_vs_N": n_sweep,
            "small_D": {"workload": f"N={N}, D=32 (4x8), L={L}, k={k}", **small}}


def suite_smalld(args):
    """Small grids (a stand-in for fields reduced to a few dozen principal components,
    Sec. 5): 75 years of D-value fields for D = 32 ... 512, L = 5, k = 20, with
    trajectory-embedded operands and with diagonal window sums. At small D the fused
    kernel's epilogue, not the contraction, sets the time; its bound is the CUDA-core
    work of the scan per output (about 8 FP32 operations: correction FMA, distance FMA,
    clamp, two compares, mask bits), reported against the FP32 ALU peak."""
    import torch

    import paper_2603_02059_gb300 as tk
    from synth import make_slp_like
    h = tk.get_handle()
    peaks, src = measured_peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    alu_peak = fp32_alu_peak_tflops(sms, float(peaks.get("sm_max_mhz", 2070.0)))
    out = []
    N, L, k, e = 27394, 5, 20, 4
    M = N - L + 1
    for gh, gw in ((4, 8), (8, 8), (8, 16), (16, 16), (16, 32)):
        X, _ = make_slp_like(N, gh, gw, seed=20260310, annual_amp=5.0)
        Xd = torch.from_numpy(X).cuda()
        row = {"D": gh * gw}
        for embed in ("always", "never"):
            h.profile_read()
            h.set_option("profile", 1)
            ms = _events_ms(lambda: tk.knn_scores(Xd, L, k, e, embed=embed, handle=h),
                            args.steps, 3)
            kms = h.profile_read()[3:]
            h.set_option("profile", 0)
            kavg = statistics.mean(kms) if kms else None
            # one evaluated output per unordered pair: M(M+1)/2 outputs
            ops = 8.0 * M * (M + 1) / 2
            row[embed] = {"ms_per_step": ms, "pairs_per_s": float(M) * M / (ms * 1e-3),
                          "kernel_ms": kavg,
                          "epilogue_alu_frac": (ops / (kavg * 1e-3) / 1e12 / alu_peak)
                          if kavg else None}
        out.append(row)
        del Xd
    if h.sync_status() != 0:
        raise RuntimeError("device-side failure")
    return {"suite": "smalld", "workload": f"N={N}, L={L}, k={k}, exclusion={e}",
            "sweep": out, "alu_peak_tflops": alu_peak, "peak_source": src}


SUITES = {"precision": suite_precision, "batched": suite_batched, "adjoint": suite_adjoint,
          "ext": suite_ext, "smalld": suite_smalld}


# --------------------------------------------------------------- reference arm

def run_reference(args, ws, rank):
    if rank != 0:
        return None
    import oracle
    from synth import config_inputs
    X, meta, cfg = config_inputs(args.workload)
    L, k, e = cfg["L"], cfg["k"], cfg["exclusion"]
    M = X.shape[0] - L + 1
    nrows = args.ref_rows
    rows_all = np.linspace(0, M - 1, nrows * (args.steps + args.warmup)).astype(np.int64)
    for w in range(args.warmup):
        oracle.knn_rows(X, L, k, e, rows_all[w * nrows:(w + 1) * nrows])
    t0 = time.perf_counter()
    for s in range(args.steps):
        r = rows_all[(args.warmup + s) * nrows:(args.warmup + s + 1) * nrows]
        oracle.knn_rows(X, L, k, e, r)
    el = (time.perf_counter() - t0) / args.steps
    value = nrows * M / el
    sample = (f"{nrows} trajectory rows x all M={M} candidates per step "
              f"(FP64 direct differences, full sort)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SLP-like anomalies)",
            "config": {"workload": (f"{args.workload}: N={X.shape[0]} days, D={X.shape[1]} "
                                    f"({meta.h}x{meta.w}), L={L}, k={k}, exclusion={e}, "
                                    f"M={M}; oracle on a bounded row sample per step")},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--fp32-steps", type=int, default=3)
    ap.add_argument("--headline", choices=["split_bf16", "bf16", "fp32"], default="split_bf16")
    ap.add_argument("--cpu-rows", type=int, default=384)
    ap.add_argument("--ref-rows", type=int, default=96)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-fp32", action="store_true", help="do not time the FP32 path")
    ap.add_argument("--skip-e2e", action="store_true", help="do not time the host-buffer path")
    ap.add_argument("--split", action="store_true",
                    help="one series shared by all ranks (strong scaling: each rank evaluates "
                         "its part of the pairs, one all-gather of candidate lists, merge)")
    ap.add_argument("--suite", choices=sorted(SUITES) + ["all"], default=None,
                    help="instead of the headline line, time the extra workloads "
                         "(one JSON line each, one GPU)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    ws, rank, local = dist_env()
    if args.suite:
        names = sorted(SUITES) if args.suite == "all" else [args.suite]
        for n in names:
            print(json.dumps(SUITES[n](args)), flush=True)
        return
    if args.impl == "reference":
        line = run_reference(args, ws, rank)
    else:
        line = run_ours(args, ws, rank, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
