#!/usr/bin/env python
"""Benchmark: greedy CSS (Algorithm 1) on the 4096 x 65536 decaying-spectrum
workload (rank 256, s_i = 1/i, noise 1e-3, k = 256), A streamed in BF16 (or
FP32) from HBM.

One step = one css_select call (initial scores + k greedy iterations) on
device-resident A.  Prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype bf16|f32]
                    [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the plain restatement of the
paper's Algorithm 1) on this machine's host cores on the same workload; each of
its steps runs two greedy iterations on the full matrix.

Multi-GPU (torchrun, one process per GPU): every rank runs its own replica of
the workload (independent problems, no collective on the data path); value is
the sum of all ranks' iterations divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import css_inputs as ci  # noqa: E402

WORKLOAD = "decay_4096x65536"
METRIC = "greedy iterations/s and achieved HBM GB/s (fused step), mixed vs plain at equal error"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--dtype", choices=["bf16", "f32"], default="bf16")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "decay_4096x32768", "dist_2048x262144", "dist_2048x65536",
                             "batched_1024", "batched_128", "relative_accuracy", "lowrank",
                             "adjoint_4096x16384"],
                    help="decay_4096x32768 is the small profiling case of the headline model; "
                         "dist_* run the distributed pipeline (Algorithms 2 and 4), batched_1024 "
                         "the batched independent problems")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-oracle", action="store_true",
                    help="skip the comparison of the headline results with the FP64 oracle "
                         "(run outside the timed region; about a minute of host time)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_array(name=WORKLOAD):
    c = ci.CONFIGS[name]
    A = ci.lowrank_decaying(c["m"], c["n"], c["rank"], c["noise"], c["seed"], dtype=np.float32)
    return c, A


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(values, device):
    """Element-wise maximum of a list of floats over all ranks (the slowest
    rank's time defines a multi-GPU step).  Identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def run_reference(args):
    """The FP64 oracle on host cores: each step = 2 iterations of Algorithm 1 on
    the full matrix (the initial scores are recomputed every step and timed
    separately)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import css_oracle as O
    c, A32 = workload_array()
    A = ci.round_bf16(A32).astype(np.float64) if args.dtype == "bf16" else A32.astype(np.float64)
    iters_per_step = 2
    for _ in range(args.warmup):
        O.greedy_css(A, 1, tau_rel=1e-6)
    it_s, tot_s, init_s = 0.0, 0.0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = O.greedy_css(A, iters_per_step, tau_rel=1e-6)
        t1 = time.perf_counter()
        tot_s += t1 - t0
        init_s += r.t_init - r.t_start
        it_s += r.t_iter[-1] - r.t_init
    value = iters_per_step * args.steps / it_s
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iterations/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": c["m"], "n": c["n"], "k": c["k"], "rank": c["rank"],
                   "noise": c["noise"], "stream_dtype": args.dtype,
                   "accumulate": "f64 throughout (the oracle; BF16 input rounded first)",
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": "iterations/s", "cores": cores, "host": host_cpu(),
                         "kind": "oracle",
                         "sample": f"{iters_per_step} iterations of Algorithm 1 per step on the full "
                                   f"{c['m']}x{c['n']} matrix in FP64; initial scores "
                                   f"{1e3 * init_s / args.steps:.0f} ms/step timed apart"},
        "e2e": {"value": value, "unit": "iterations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def host_cpu():
    """The host's CPU model and architecture, for the CPU baseline's record
    (lscpu where it is installed, else /proc/cpuinfo)."""
    import platform
    name = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not name:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        name = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return f"{name or 'unknown model'} ({platform.machine()})"


def cpu_baseline(A32, dtype):
    """Oracle on a bounded sample: 3 iterations of Algorithm 1 on the full matrix
    (FP64), iterations timed apart from the initial scores."""
    from oracle import css_oracle as O
    A = ci.round_bf16(A32).astype(np.float64) if dtype == "bf16" else A32.astype(np.float64)
    r = O.greedy_css(A, 3, tau_rel=1e-6)
    it = r.t_iter[-1] - r.t_init
    return {"value": 3 / it, "unit": "iterations/s", "cores": os.cpu_count(), "host": host_cpu(),
            "kind": "oracle",
            "sample": f"3 iterations of Algorithm 1 on the full {A.shape[0]}x{A.shape[1]} matrix in "
                      f"FP64 (initial scores {r.t_init - r.t_start:.1f} s, timed apart)"}


def _events(torch, n):
    return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(n)]


def run_distributed(args):
    """Algorithm 2 then Algorithm 4 on 2048 x n BF16 (rank 400 + 1e-3 noise):
    B = A Omega on tensor cores, 64 log-normal column blocks selecting 100
    each by GCSS, GCSS on the union for k = 100.  One step = the pipeline."""
    import torch
    from paper_1312_6838_gb300 import css
    c = dict(ci.CONFIGS["dist_2048x262144"])
    if args.workload == "dist_2048x65536":
        c["n"] = 65536
        c["blocks"] = 16
    m, n, r = c["m"], c["n"], c["r"]
    A32 = ci.lowrank_decaying(m, n, c["rank"], c["noise"], c["seed"], dtype=np.float32)
    A = torch.from_numpy(np.ascontiguousarray(A32.T)).cuda().to(torch.bfloat16).t()
    del A32
    Om = torch.from_numpy(np.ascontiguousarray(
        ci.gaussian_omega(n, r, c["omega_seed"]).T)).cuda().to(torch.bfloat16).t()
    offs = ci.lognormal_blocks(n, c["blocks"], c["block_median"], c["block_sigma"],
                               c["block_seed"]).tolist()
    def step():
        B = css.project(A, Om)
        return B, css.distributed(A, B, offs, c["l_block"], c["k"])
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    ev = _events(torch, args.steps)
    evp = _events(torch, args.steps)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        ev[i][0].record()
        evp[i][0].record()
        B = css.project(A, Om)
        evp[i][1].record()
        res = css.distributed(A, B, offs, c["l_block"], c["k"])
        ev[i][1].record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    tot = [a.elapsed_time(b) for a, b in ev]
    proj = [a.elapsed_time(b) for a, b in evp]
    # the projection with Omega drawn on the device instead of read from HBM:
    # Gaussian (generated, then the tensor-core product) and the sparse random
    # sign matrix (no Omega formed), Sec. 5.1 / Sec. 7's "rnd" and "ssgn"
    def t_ms(f, reps=5):
        f()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            f()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    proj_gen = t_ms(lambda: css.project_random(A, r, c["omega_seed"], "gaussian"))
    proj_ssgn = t_ms(lambda: css.project_random(A, r, c["omega_seed"], "sparse_sign"))
    block_iters = int((res.block_sel >= 0).sum().item())
    iters = block_iters + res.n_sel
    ms = statistics.mean(tot)
    pms = statistics.mean(proj)
    # the blocks' persistent launch timed on its own (CUDA events inside the
    # call): per block iteration it streams the block's columns once and
    # reads and writes their score state; one more pass forms g^(0)
    B = css.project(A, Om)
    phases = []
    for _ in range(3):
        tl = []
        css.distributed(A, B, offs, c["l_block"], c["k"], timing=tl)
        phases.append(tl)
    init_ms = statistics.mean(p[0] for p in phases)
    block_ms = statistics.mean(p[1] for p in phases)
    widths = np.diff(np.asarray(offs))
    kbs = np.minimum(c["l_block"], widths)
    block_bytes = float(np.sum((kbs + 1) * widths * m * 2 + kbs * 48 * widths))
    block_gbs = block_bytes / (block_ms / 1e3) / 1e9
    hbm_peak, hbm_kind = peaks()
    peak_tf = 1845.9
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak_tf = float(json.load(fh)["bf16_tflops"])
    except Exception:
        pass
    tf = 2.0 * m * n * r / (pms / 1e3) / 1e12
    print(json.dumps({
        "metric": "greedy iterations/s of the distributed pipeline (Algorithms 2 and 4)",
        "value": iters / (ms / 1e3), "unit": "iterations/s", "n_gpus": 1, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": args.workload, "m": m, "n": n, "r": r, "blocks": len(offs) - 1,
                   "l_block": c["l_block"], "k": c["k"], "block_iterations": block_iters},
        "projection_ms": pms,
        "projection_generated_gaussian_ms": proj_gen,
        "projection_sparse_sign_ms": proj_ssgn,
        "initial_scores_ms": init_ms,
        "block_phase_ms": block_ms,
        # traffic: DRAM bytes read + written by the blocks' launch, from an
        # ncu capture on the 2048 x 65536 case (16 blocks, the kernel's
        # two-CTAs-per-SM shape): 26.984 GB for 27.427 GB algorithmic, scaled
        # by this launch's algorithmic bytes
        "roofline": {"bound": "hbm", "achieved": block_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": block_gbs / hbm_peak,
                     "traffic": block_bytes * (26.947826176e9 + 0.036115200e9) / 27.426553856e9,
                     "peak_kind": hbm_kind,
                     "kernel": "greedy_kernel (the 64 blocks' persistent launch, Algorithm 4's map phase)",
                     "bytes_per_launch": block_bytes,
                     "bytes": "per block: (l_b + 1) passes over its columns in BF16 + 48 B of score "
                              "state per column and iteration; B's reads (L2-resident) not counted"},
        "roofline_projection": {"bound": "tensor", "achieved": tf, "peak": peak_tf, "unit": "TFLOP/s",
                                "frac": tf / peak_tf, "traffic": None, "kernel": "tc_kernel (B = A Omega)"},
        # per pipeline: projection (tensor-core partials, reduction), the
        # blocks' initial scores (split of B, tensor-core column norms), the
        # blocks' greedy launch, the union on the device (scan, global ids,
        # gather of columns and of scores), the union's greedy launch, the
        # final picks' global ids
        "gpu_launches": 11 * args.steps, "clocks": clk}), flush=True)


def run_batched(args):
    """1024 independent instances (FP32, rank k + 1e-2 noise): one persistent
    launch (FP32 and BF16 streams) against a loop of single-instance calls."""
    import torch
    from paper_1312_6838_gb300 import css
    c = ci.CONFIGS[args.workload]
    specs = ci.batched_specs(c["count"], c["seed"])
    As32, ks = [], []
    for i, (m, n, k) in enumerate(specs):
        A = ci.batched_instance(m, n, k, c["seed"] + i, noise=c["noise"])
        As32.append(torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t())
        ks.append(k)
    As16 = [css.to_colmajor(a.to(torch.bfloat16)) for a in As32]
    total_k = sum(ks)
    def t_ms(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps
    ph32, ph16 = [], []
    css.select_batched(As32, ks, timing=ph32)
    css.select_batched(As16, ks, timing=ph16)
    clocks = ClockSampler(0)
    clocks.start()
    ms32 = t_ms(lambda: css.select_batched(As32, ks))
    ms16 = t_ms(lambda: css.select_batched(As16, ks))
    loop32 = t_ms(lambda: [css.select(a, k) for a, k in zip(As32, ks)])
    clk = clocks.stop()
    # equal final error (outside the timed region): every instance's BF16
    # batched selection and its FP32 single-call selection, both evaluated
    # directly on the FP32 matrix (the residual formed on the device, FP64
    # sum); the FP32 batched selections are compared the same way, to show
    # how far near-tie picks alone move the error of these problems
    r16, r32 = [], []
    for a, k, b16, b32 in zip(As32, ks, css.select_batched(As16, ks), css.select_batched(As32, ks)):
        e_plain = css.residual_error(a, css.select(a, k).indices)
        r16.append(css.residual_error(a, b16.indices) / e_plain)
        r32.append(css.residual_error(a, b32.indices) / e_plain)

    def summary(r):
        r = np.asarray(r)
        return {"min": float(r.min()), "median": float(np.median(r)), "max": float(r.max()),
                "geomean": float(np.exp(np.mean(np.log(r)))),
                "within_1pct": float(np.mean(np.abs(r - 1.0) <= 0.01)),
                "within_1e-4": float(np.mean(np.abs(r - 1.0) <= 1e-4))}
    # roofline of the BF16 batched persistent launch: per problem, k + 1
    # passes over its BF16 columns, C = A A^T (FP32) read once per iteration,
    # and the score state
    greedy_ms16 = ph16[1]
    batch_bytes = float(sum((k + 1) * m * n * 2 + k * (m * m * 4 + 48 * n) for (m, n, k) in specs))
    batch_gbs = batch_bytes / (greedy_ms16 / 1e3) / 1e9
    hbm_peak, hbm_kind = peaks()
    # the FP64 oracle on a seeded sample of the problems (outside the timed
    # region): each batched selection's error against the oracle's selection
    # on the same values (BF16-rounded for the BF16 batch), and the oracle's
    # own rate on the host cores
    from oracle import css_oracle as O
    rng = np.random.default_rng(2024)
    sample = rng.choice(len(specs), size=48, replace=False)
    b16_all = css.select_batched(As16, ks)
    b32_all = css.select_batched(As32, ks)
    o16, o32 = [], []
    t_or, k_or = 0.0, 0
    for i in sample:
        v32 = As32[i].cpu().numpy().astype(np.float64)
        v16 = As16[i].float().cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        ref16 = O.greedy_css(v16, ks[i], tau_rel=1e-6)
        t_or += time.perf_counter() - t0
        k_or += len(ref16.S)
        ref32 = O.greedy_css(v32, ks[i], tau_rel=1e-6)
        o16.append(O.reconstruction_error(v16, b16_all[i].indices.cpu().tolist())
                   / O.reconstruction_error(v16, ref16.S))
        o32.append(O.reconstruction_error(v32, b32_all[i].indices.cpu().tolist())
                   / O.reconstruction_error(v32, ref32.S))
    print(json.dumps({
        "metric": f"greedy iterations/s, {len(specs)} independent problems",
        "value": total_k / (ms16 / 1e3), "unit": "iterations/s", "n_gpus": 1, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms16, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": args.workload, "instances": len(ks), "total_k": total_k,
                   "sum_mn": int(sum(m * n for m, n, _ in specs))},
        "batched_fp32_iterations_per_s": total_k / (ms32 / 1e3),
        "loop_fp32_iterations_per_s": total_k / (loop32 / 1e3),
        "speedup_batched_bf16_vs_loop_fp32": loop32 / ms16,
        "speedup_batched_fp32_vs_loop_fp32": loop32 / ms32,
        "phases_ms_fp32": {"initial_scores": ph32[0], "greedy": ph32[1]},
        "phases_ms_bf16": {"initial_scores": ph16[0], "greedy": ph16[1]},
        "equal_error": {"bf16_batched_over_fp32_loop": summary(r16),
                        "fp32_batched_over_fp32_loop": summary(r32),
                        "evaluated": "per instance, the ratio of ||A - P_S A||_F^2 of a batched "
                                     "selection to that of the FP32 single-call selection, both formed "
                                     "directly on the FP32 matrix (css.residual_error)"},
        "oracle": {"bf16_batched_over_oracle": summary(o16), "fp32_batched_over_oracle": summary(o32),
                   "sample": "48 seeded problems; each batched selection's error over the FP64 oracle's "
                             "selection's error, both on the values the device holds (FP64, "
                             "reconstruction_error)"},
        # DRAM traffic per launch: the ncu capture of the BF16 launch of the
        # 128-problem case of the same model read and wrote 1.064 x its
        # algorithmic bytes (each C = A A^T comes from DRAM every iteration,
        # as counted), scaled by the bytes of this launch
        "roofline": {"bound": "hbm", "achieved": batch_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": batch_gbs / hbm_peak, "traffic": 1.064 * batch_bytes, "peak_kind": hbm_kind,
                     "kernel": f"greedy_kernel (all {len(specs)} problems in one persistent launch, BF16)",
                     "bytes_per_launch": batch_bytes,
                     "bytes": "per problem: (k + 1) passes over A in BF16, C = A A^T (FP32) read "
                              "once per iteration, 48 B of score state per column and iteration"},
        "cpu_baseline": {"value": k_or / t_or, "unit": "iterations/s", "cores": os.cpu_count(),
                         "host": host_cpu(), "kind": "oracle",
                         "sample": "Algorithm 1 in FP64 on the 48 sampled problems' BF16 values, "
                                   "initial scores included"},
        # per BF16 batch: the copy of A to aligned buffers (these leading
        # dimensions are not multiples of 8), C = A A^T, its chunk sum and
        # mirror, the split of C, column dots, row sums (one grouped launch
        # each over all problems) + the persistent greedy kernel
        "gpu_launches": 7 * args.steps,
        "clocks": clk}), flush=True)


def run_relative_accuracy(args):
    """The evaluation measure of Sec. 7 on a synthetic matrix with a decaying
    spectrum (2048 x 16384 BF16, rank 400 + 1e-3 noise): GreedyCSS,
    RndGreedyCSS (Gaussian and sparse sign Omega) and the distributed
    selection (Algorithms 2 and 4, 16 blocks) against uniform sampling without
    replacement (mean error over 10 seeds, 0 %) and the best rank-l
    approximation (FP64 SVD of the same BF16 values, 100 %).  Errors
    ||A - P_S A||_F come from the device (css_residual_backward, loss only)."""
    import torch
    from paper_1312_6838_gb300 import css
    m, n, rank = 2048, 16384, 400
    A32 = ci.lowrank_decaying(m, n, rank, 1e-3, 3, dtype=np.float32)
    A = torch.from_numpy(np.ascontiguousarray(A32.T)).cuda().to(torch.bfloat16).t()
    vals = A.float().cpu().numpy().astype(np.float64)
    del A32
    # best rank-l errors from the eigenvalues of A A^T (FP64)
    ev = np.sort(np.clip(np.linalg.eigvalsh(vals @ vals.T), 0.0, None))[::-1]
    fro2 = float(np.sum(vals * vals))

    def err(S):
        return float(np.sqrt(max(css.residual(A, list(S)).item(), 0.0)))

    def timed(f):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = f()
        torch.cuda.synchronize()
        return out, (time.perf_counter() - t0) * 1e3

    offs = [int(x) for x in np.linspace(0, n, 17)]
    rows = {}
    for l in (16, 64, 128):
        e_svd = float(np.sqrt(max(fro2 - ev[:l].sum(), 0.0)))
        rng = np.random.default_rng(100 + l)
        e_uni = float(np.mean([err(rng.choice(n, l, replace=False)) for _ in range(10)]))
        css.select(A, l)                                   # first launches outside timing
        methods = {
            "GreedyCSS": lambda: css.select(A, l).indices.cpu().tolist(),
            "RndGreedyCSS (rnd)": lambda: css.select_randomized(A, l, 5, "gaussian").indices.cpu().tolist(),
            "RndGreedyCSS (ssgn)": lambda: css.select_randomized(A, l, 5, "sparse_sign").indices.cpu().tolist(),
            "DistGreedyCSS (rnd, 16 blocks)": lambda: css.distributed(
                A, css.project_random(A, l, 5, "gaussian"), offs, max(1, l // 4), l).indices.cpu().tolist(),
        }
        row = {"l": l, "svd_error": e_svd, "uniform_error": e_uni}
        for name, f in methods.items():
            S, ms = timed(f)
            e = err(S)
            row[name] = {"relative_accuracy_pct": 100.0 * (e_uni - e) / (e_uni - e_svd), "error": e,
                         "ms": ms}
        rows[str(l)] = row
    best = rows["64"]["GreedyCSS"]["relative_accuracy_pct"]
    print(json.dumps({
        "metric": "relative accuracy (%) of GreedyCSS at l = 64 (Sec. 7's measure)", "value": best,
        "unit": "%", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
        "config": {"workload": "relative_accuracy", "m": m, "n": n, "rank": rank, "noise": 1e-3,
                   "dtype": "bf16", "uniform_seeds": 10},
        "results": rows}), flush=True)


FP64_TFLOPS = 1.20   # FP64 FMA throughput of this part, measured with a dependent-free FMA loop
FP32_TFLOPS = 67.9   # FP32 FMA throughput of this part, measured the same way


def run_adjoint(args):
    """The adjoint of the reconstruction error at a fixed selected set: A
    4096 x 16384 FP32 (rank 128 + 1e-3 noise), S = the device's greedy
    selection of 128 columns; each timed step is one css_residual_backward
    call forming the loss and dA (the backward of css.residual).  A (268 MB)
    and dA are larger than L2."""
    import torch
    import ctypes as C
    from paper_1312_6838_gb300 import css, _lib as L
    c = ci.CONFIGS["adjoint_4096x16384"]
    m, n, k = c["m"], c["n"], c["k"]
    A32 = ci.lowrank_uv(m, n, c["rank"], c["noise"], c["seed"], dtype=np.float32)
    A = css.to_colmajor(torch.from_numpy(A32).cuda())
    S = css.select(A, k).indices
    lib = L.load()
    dA = css.empty_colmajor(m, n, torch.float32, "cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    o = L.default_opts()
    nbytes = lib.css_workspace_size(L.CSS_OP_BACKWARD, L.CSS_F32, m, n, 0, k, 0, C.byref(o))
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    off = (-buf.data_ptr()) % 256
    ws = buf[off:off + nbytes]
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def step():
        code = lib.css_residual_backward(C.c_void_p(A.data_ptr()), L.CSS_F32, m, n, m, C.c_void_p(S.data_ptr()), k,
                                         1.0, C.c_void_p(dA.data_ptr()), m, C.c_void_p(loss.data_ptr()),
                                         C.c_void_p(ws.data_ptr()), nbytes, C.byref(o), stream)
        assert code == 0, code

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    clk = ClockSampler(0)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    flop = 6.0 * k * m * n          # Q^T A, A - Q W, R W^T: 2 k m n each
    tf = flop / (ms * 1e-3) / 1e12
    line = {
        "metric": "adjoint of ||A - P_S A||_F^2 at fixed S: loss and dA per call",
        "value": ms, "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": ms, "higher_is_better": False, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "adjoint_4096x16384", "m": m, "n": n, "k": k, "rank": c["rank"],
                   "noise": c["noise"], "l2": "A and dA (268 MB each) larger than L2"},
        "roofline": {"bound": "alu", "achieved": tf, "peak": FP32_TFLOPS, "unit": "TFLOP/s",
                     "frac": tf / FP32_TFLOPS, "traffic": None,
                     "kernel": "the adjoint's three GEMM-shaped kernels (double-float W and R, FP32 R W^T)",
                     "note": "algorithmic 6 k m n FLOPs; W and R run in double-float (about 12 FP32 operations "
                             "per multiply-add), so the FP32 pipe does several times the algorithmic count"},
        "hbm_bytes_per_call": 3 * m * n * 4, "loss": float(loss.item()), "clocks": clocks,
        # per call: gather A_S, Gram (2), the Cholesky (one launch for
        # k <= 128; above, the blocked form: initial diagonal, per 32-column
        # panel the diagonal block and, but for the last panel, the rows below
        # and the trailing update), L^-1, Q, W, R with the loss partials, loss
        # sum, R W^T slices, their sum, dA_S
        "gpu_launches": (12 if k <= 128 else 10 + 3 * ((k + 31) // 32)) * args.steps,
    }
    if not args.no_cpu_baseline:
        from oracle import css_oracle as O
        vals = A32.astype(np.float64)
        Sl = S.cpu().tolist()
        t0 = time.perf_counter()
        L_ref, _ = O.residual_gradient(vals, Sl)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": dt * 1e3, "unit": "ms", "cores": os.cpu_count(), "host": host_cpu(),
                                "kind": "oracle",
                                "sample": "one full call (closed-form FP64 gradient, numpy on the host)"}
        line["loss_rel_diff_vs_oracle"] = abs(line["loss"] - L_ref) / L_ref
    print(json.dumps(line), flush=True)


def run_lowrank(args):
    """Sec. 3.2 after the headline selection: the greedy run on the
    4096 x 65536 BF16 workload (k = 256, basis and omega rows kept), then the
    rank-128 approximation and approximate SVD from that embedding
    (css_lowrank: Gram matrix, Jacobi eigendecomposition, U~ and V~).  Each
    timed step is one css_lowrank call; W (134 MB) is larger than L2."""
    import torch
    from paper_1312_6838_gb300 import css
    c, A32 = workload_array(WORKLOAD)
    m, n, k = c["m"], c["n"], c["k"]
    kr = 128
    A = css.to_colmajor(torch.from_numpy(A32).cuda().to(torch.bfloat16))
    del A32
    res = css.select(A, k, return_W=True, return_basis=True)
    W, Q = res.W, res.basis
    l = res.n_sel
    for _ in range(max(args.warmup, 3)):
        css.lowrank(W, kr, Q)
    phases = css.lowrank(W, kr, Q, timing=True).timing_ms
    # the embedding of Sec. 3.2 formed from scratch for the same selection
    # (CholeskyQR2 of A_S, then W = Q^T A in double-float arithmetic)
    S = res.indices
    css.embed(A, S)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(2):
        css.embed(A, S)
    e1.record()
    torch.cuda.synchronize()
    embed_ms = e0.elapsed_time(e1) / 2
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(0)
    clk.start()
    ev0.record()
    for _ in range(args.steps):
        out = css.lowrank(W, kr, Q)
    ev1.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    # the dominant kernel: the Gram matrix W W^T, l (l + 1) / 2 n FP64 FMAs
    gram_flop = 2.0 * (l * (l + 1) / 2) * n
    gram_tf = gram_flop / (phases[0] * 1e-3) / 1e12
    v_flop = 2.0 * n * l * kr + 2.0 * m * l * kr
    line = {
        "metric": "rank-k approximation and approximate SVD from the embedding (Sec. 3.2)",
        "value": ms, "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": ms, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"lowrank_{WORKLOAD}", "m": m, "n": n, "l": l, "k": kr,
                   "selection_dtype": "bf16", "l2": "W (134 MB) larger than L2"},
        "phases_ms": {"gram": phases[0], "eigendecomposition": phases[1], "products": phases[2]},
        "jacobi_sweeps": int(phases[3]),
        "embed_ms": embed_ms,
        # algorithmic FLOP rates: the Gram matrix in FP64, the products of
        # FP64 operands accumulated in double-float on the FP32 pipe
        "tflops": {"gram_fp64": gram_tf,
                   "products_double_float": v_flop / (phases[2] * 1e-3) / 1e12},
        # traffic: DRAM bytes read + written by one gram_rows_kernel launch on
        # this workload, from an ncu capture of that kernel (W read once, the
        # slices' partial tiles written)
        "roofline": {"bound": "alu", "achieved": gram_tf, "peak": FP64_TFLOPS, "unit": "TFLOP/s",
                     "frac": gram_tf / FP64_TFLOPS,
                     "traffic": (134.7e6 + 9.4e6) if (m, n, l) == (4096, 65536, 256) else None,
                     "kernel": "gram_rows_kernel (FP64)"},
        "sigma_1": float(out.sigma[0]), "tail": out.tail, "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        from oracle import css_oracle as O
        Wn, Qn = W.cpu().numpy(), Q.cpu().numpy()
        t0 = time.perf_counter()
        ref = O.rank_k_approximation(Qn, Wn, kr)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": dt * 1e3, "unit": "ms", "cores": os.cpu_count(), "host": host_cpu(),
                                "kind": "oracle",
                                "sample": "the whole problem once (numpy/LAPACK thin SVD of W)"}
        line["max_sigma_rel_diff_vs_oracle"] = float(
            np.max(np.abs(out.sigma.cpu().numpy() - ref["sigma"]) / ref["sigma"]))
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload.startswith("dist_"):
        run_distributed(args)
        return
    if args.workload.startswith("batched_"):
        run_batched(args)
        return
    if args.workload == "relative_accuracy":
        run_relative_accuracy(args)
        return
    if args.workload == "lowrank":
        run_lowrank(args)
        return
    if args.workload == "adjoint_4096x16384":
        run_adjoint(args)
        return
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_1312_6838_gb300 import css
    from paper_1312_6838_gb300 import _lib

    c, A32 = workload_array(args.workload)
    m, n, k = c["m"], c["n"], c["k"]
    tdt = torch.bfloat16 if args.dtype == "bf16" else torch.float32
    # column-major: the (n, m) row-major storage of A^T
    At_host = torch.from_numpy(np.ascontiguousarray(A32.T))
    A = At_host.to(dev).to(tdt).t()
    assert A.stride(0) == 1 and A.shape == (m, n)
    a_bytes = m * n * A.element_size()
    c_bytes = m * m * 4

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        css.select(A, k)
    stream = torch.cuda.current_stream()
    barrier()
    clocks = ClockSampler(local if ws > 1 else 0)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    init_ms, loop_ms = [], []
    barrier()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        ev[i][0].record(stream)
        res = css.select(A, k, timing=True)
        ev[i][1].record(stream)
        init_ms.append(res.timing_ms[0])
        loop_ms.append(res.timing_ms[1])
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(step_ms)
    tot_loop = sum(loop_ms)
    tot_ms, tot_loop = max_over_ranks([tot_ms, tot_loop], dev)
    iters = ws * args.steps * res.n_sel
    value = iters / (tot_loop / 1e3)
    # roofline of the persistent greedy kernel: per iteration it streams A once,
    # reads C = A A^T once and reads/writes the score state (f, g: r+w, g0: r, W: w)
    per_iter = a_bytes + c_bytes + 48 * n
    achieved = per_iter * res.n_sel / (statistics.mean(loop_ms) / 1e3) / 1e9
    # DRAM traffic per launch from an ncu capture of the greedy kernel on the
    # 4096 x 32768 case of the same model (17 A passes): reads 1.0153 x the
    # bytes of A and writes 57 B per column per A pass (C stays in L2),
    # scaled by the A passes of this launch
    traffic = None
    if args.workload in (WORKLOAD, "decay_4096x32768") and args.dtype == "bf16":
        traffic = (res.n_sel + 1) * (a_bytes * 1.0153 + 57.3 * n)
    peak, peak_kind = peaks()
    out = {
        "metric": METRIC, "value": value, "unit": "iterations/s", "n_gpus": ws,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": tot_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": args.workload, "m": m, "n": n, "k": k, "rank": c["rank"],
                   "noise": c["noise"], "stream_dtype": args.dtype,
                   "accumulate": "f32 dot products, f64 score state and basis",
                   "l2": f"inputs larger than L2 (A = {a_bytes / 2**20:.0f} MiB per pass)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "init_ms": statistics.mean(init_ms), "loop_ms": statistics.mean(loop_ms),
        "whole_call_iterations_per_s": ws * args.steps * res.n_sel / (tot_ms / 1e3),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "greedy_kernel (persistent: pivot phases + fused step)",
                     "bytes_per_iteration": per_iter, "peak_kind": peak_kind},
        # per css_select: C = A A^T (lower tiles), its chunk sum and mirror,
        # the split of C, column dots, row sums (tensor cores; FP32 A is
        # split into parts first) + the persistent greedy kernel
        "gpu_launches": (6 if args.dtype == "bf16" else 7) * args.steps,
        "clocks": clk,
    }
    out["hbm_gbs"] = achieved
    # the end-to-end leg first: the oracle legs below keep the host's cores
    # busy (multithreaded BLAS), which the host-driven e2e timing would see
    if not args.no_e2e:
        out["e2e"] = e2e(css, A32, tdt, m, n, k, dev, args)
    S_timed = res.indices.cpu().tolist()
    if rank == 0 and not args.no_oracle and args.workload in (WORKLOAD, "decay_4096x32768"):
        out["oracle"] = {args.dtype: oracle_comparison(css, A, A32, args.dtype, k, S_timed)}
    if args.dtype == "bf16" and args.workload in (WORKLOAD, "decay_4096x32768"):
        del A
        pc = plain_comparison(css, At_host, dev, k, c_bytes, n, S_timed)
        S_plain = pc.pop("_S_plain")
        out.update(pc)
        if rank == 0 and not args.no_oracle:
            A = At_host.to(dev).t()
            out["oracle"]["f32"] = oracle_comparison(css, A, A32, "f32", k, S_plain)
            del A
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(A32, args.dtype)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def plain_comparison(css, At_host, dev, k, c_bytes, n, S_mixed):
    """The plain path beside the mixed one (outside the timed region): the
    same selection with A streamed in FP32, its greedy-loop rate and HBM
    rate, and both selections' reconstruction errors formed directly on the
    FP32 matrix."""
    A = At_host.to(dev).t()
    a_bytes = A.shape[0] * A.shape[1] * 4
    for _ in range(2):
        css.select(A, k)
    loop = []
    for _ in range(3):
        r = css.select(A, k, timing=True)
        loop.append(r.timing_ms[1])
    ms = statistics.mean(loop)
    e_plain = css.residual_error(A, r.indices)
    e_mixed = css.residual_error(A, S_mixed)
    S_plain = r.indices.cpu().tolist()
    del A
    return {
        "_S_plain": S_plain,
        "plain_f32": {"value": r.n_sel / (ms / 1e3), "unit": "iterations/s", "loop_ms": ms,
                      "hbm_gbs": (a_bytes + c_bytes + 48 * n) * r.n_sel / (ms / 1e3) / 1e9},
        "equal_error": {"mixed_bf16": e_mixed, "plain_f32": e_plain,
                        "rel_diff": abs(e_mixed - e_plain) / e_plain,
                        "evaluated": "||A - P_S A||_F^2 of each selection formed directly on the FP32 "
                                     "matrix (css.residual_error)"},
    }


def oracle_comparison(css, A, A32, dtype, k, S_dev):
    """The result against the FP64 oracle, outside the timed region.

    The oracle (Algorithm 1 in FP64 on the values the device holds) selects
    its own k columns.  The device is then run once with the oracle's whole
    sequence forced and reports its own argmax at every iteration: steps
    that agree, and mismatches split by the oracle's top-two gap (at most
    1e-6: both picks correct under the 1e-6 rule; above it: decided inside
    the mixed path's score error).  Where the device's own selection parts
    from the oracle's, the oracle is re-run forced on the device's sequence
    and every device pick is checked against the best score on its own path
    (tests/gpu_helpers.py, certify_selection).  Both selections' errors
    ||A - P_S A||_F^2 are formed in FP64 on the same values."""
    from oracle import css_oracle as O
    from tests.gpu_helpers import certify_selection
    import torch
    vals = ci.round_bf16(A32).astype(np.float64) if dtype == "bf16" else A32.astype(np.float64)
    m = vals.shape[0]
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    t0 = time.perf_counter()
    ref = O.greedy_css(vals, k, tau_rel=1e-6, keep_scores=True)
    forced = css.select(A, len(ref.S), forced=list(ref.S), diag=True)
    own = forced.diag_argmax.cpu().tolist()
    mism = [(t, float(ref.gaps[t])) for t in range(len(ref.S)) if own[t] != ref.S[t]]
    strict = [g for _, g in mism if g <= 1e-6]
    wide = [g for _, g in mism if g > 1e-6]
    del ref.scores[:], ref.fs[:], ref.gs[:]
    e_dev = O.reconstruction_error(vals, S_dev, chunk=8192)
    e_ref = O.reconstruction_error(vals, ref.S, chunk=8192)
    first = next((t for t in range(min(len(S_dev), len(ref.S))) if S_dev[t] != ref.S[t]), None)
    line = {
        "oracle_steps": len(ref.S),
        "steps_agreeing_on_oracle_path": len(ref.S) - len(mism),
        "mismatches_gap_le_1e-6": len(strict),
        "mismatches_gap_gt_1e-6": len(wide),
        "largest_gap_of_a_mismatch": max([g for _, g in mism], default=0.0),
        "mismatch_steps": mism,
        "error_device_selection": e_dev,
        "error_oracle_selection": e_ref,
        "relative_difference": (e_dev - e_ref) / e_ref,
        "first_step_own_selection_parts": first,
        "common_columns": len(set(S_dev) & set(ref.S)),
    }
    if first is not None:
        on_dev = O.greedy_css(vals, len(S_dev), tau_rel=1e-6, keep_scores=True, forced=S_dev)
        try:
            n_off, worst = certify_selection(S_dev, on_dev, m, tdt)
            line["own_selection_certified"] = True
            line["own_selection_picks_off_argmax"] = n_off
            line["own_selection_largest_deficit"] = worst
        except AssertionError as exc:
            line["own_selection_certified"] = False
            line["own_selection_failure"] = str(exc)[:200]
    line["host_seconds"] = time.perf_counter() - t0
    return line


def e2e(css, A32, tdt, m, n, k, dev, args):
    """Same metric through the public C-ABI host entry point: pinned host A ->
    device copy -> selection -> results back to the host, all timed."""
    import torch
    A_host = torch.from_numpy(np.ascontiguousarray(A32.T)).to(tdt).pin_memory().t()
    A_dev = css.empty_colmajor(m, n, tdt, dev)
    nbytes = css.host_workspace_bytes(m, n, k, tdt)
    _buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    off = (-_buf.data_ptr()) % 256
    wsb = _buf[off:off + nbytes]
    for _ in range(2):
        css.select_host(A_host, k, A_dev, ws=wsb)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ns = 0
    for _ in range(args.steps):
        sel, trace, n_sel = css.select_host(A_host, k, A_dev, ws=wsb)
        ns += n_sel
    dt = time.perf_counter() - t0
    return {"value": ns / dt, "unit": "iterations/s",
            "h2d_bytes_per_step": m * n * A_host.element_size(),
            "d2h_bytes_per_step": 4 * k + 8 * (k + 1) + 4,
            "note": "initial scores included (whole call)"}


if __name__ == "__main__":
    main()
