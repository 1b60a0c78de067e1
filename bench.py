#!/usr/bin/env python
"""Benchmark of C = A^t A on one GB300 (or N replicas under torchrun).

Default workload: ATA at the paper's scale with FP64 accuracy, A 10000 x 10000
FP64 with i.i.d. N(0, 1) entries from seed 1, leaves emulating FP64 on the
bf16 tensor cores (6 slices), cutoff chosen by the planner's autotuner, packed
upper-triangle FP64 output, componentwise error against the oracle <= 1e-11;
the plain FP64 path on the same input is timed beside it.  A step is one
ata_execute (one replay of the plan's CUDA graph: operand splits, operand
preparation, the persistent leaf launch, Strassen combines) over the resident
input.  The metric is effective TFLOP/s = 2 m n^2 / t (m n^2 classical FMAs),
at the error reported in the line.  Other workloads: --workload NAME (the
plain FP64 and precision forms, batched, serving, and the general product
C = X^t Y through ata_gemm_tn, metric 2 m p r / t).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME]

--impl reference times the test oracle (plain FP64 triple loop, OpenMP on the
host cores) on a bounded sample of the same workload, extrapolated to the
whole product.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (m, n, leaf mode, generator, seed, cutoff (0 = autotune))
    # paper scale, FP64 input, 1e-11 componentwise: plain FP64 leaves ...
    "ata_f64_10000x10000": (10000, 10000, "f64", "normal", 1, 0),
    "ata_f64_5000x5000": (5000, 5000, "f64", "normal", 1, 0),
    "ata_f64_20000x8000": (20000, 8000, "f64", "normal", 1, 0),
    # ... and FP64-accurate leaves emulated on bf16 tensor cores
    "ata_ozaki_10000x10000": (10000, 10000, "ozaki", "normal", 1, 0),
    "ata_ozaki_5000x5000": (5000, 5000, "ozaki", "normal", 1, 0),
    "ata_ozaki_20000x8000": (20000, 8000, "ozaki", "normal", 1, 0),
    # precision form: FP32 16384 x 8192, every 8th column x 1e3
    "ata_bf16x3_16384x8192": (16384, 8192, "bf16x3", "scaled_cols", 2, 0),
    "ata_tf32_16384x8192": (16384, 8192, "tf32", "scaled_cols", 2, 0),
    "ata_f64_512x384": (512, 384, "f64", "uniform", 0, 64),
    # small cases for ncu captures (A larger than L2, a few GB on the device)
    "ata_f64_4500x4500_c600": (4500, 4500, "f64", "normal", 1, 600),
    "ata_ozaki_4500x4500_c1200": (4500, 4500, "ozaki", "normal", 1, 1200),
    "ata_bf16x3_8192x4096_c1024": (8192, 4096, "bf16x3", "scaled_cols", 2, 1024),
    "ata_tf32_8192x4096_c1024": (8192, 4096, "tf32", "scaled_cols", 2, 1024),
}
MODE_CODES = {"f64": 0, "bf16x3": 1, "tf32": 2, "ozaki": 3}
PAIRS = {"f64": 1, "bf16x3": 6, "tf32": 1, "ozaki": 21}
TOLERANCE = {"f64": ("componentwise", 1e-11), "ozaki": ("componentwise", 1e-11),
             "bf16x3": ("normwise", 1e-6), "tf32": ("normwise", 1e-3)}
DEFAULT_WORKLOAD = "ata_ozaki_10000x10000"
# general product C = X^t Y (X: m x p, Y: m x r): the top C_12 product of a
# 10000^2 A^t A, and the precision form's shape
GEMM_WORKLOADS = {
    # name: (m, p, r, leaf mode, generator, seed, cutoff (0 = autotune))
    "gemm_tn_ozaki_10000x5000x5000": (10000, 5000, 5000, "ozaki", "normal", 1, 0),
    "gemm_tn_f64_10000x5000x5000": (10000, 5000, 5000, "f64", "normal", 1, 0),
    "gemm_tn_bf16x3_16384x4096x4096": (16384, 4096, 4096, "bf16x3", "scaled_cols", 2, 0),
}
# workloads run by their own drivers (not single products)
EXTRA_WORKLOADS = ["batched_bf16x3", "batched_f64", "serving_bf16x3", "serving_ozaki", "serving_f64"]

# Peak of the FP64 leaf arithmetic: 2 DFMA per clock per SM (the step-0
# probe measured 1.204 TFLOP/s of DFMA on 152 SMs) at the 2070 MHz maximum
# SM clock: 152 * 2 * 2 FLOP * 2.07e9 = 1.2586 TFLOP/s.
FP64_ALU_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# Tensor peaks: the measured cuBLAS bf16 burst figure (MEASURED_PEAKS.json
# bf16_tflops, 1886.9 TFLOP/s when this was written); TF32 is that figure
# times the nominal tf32/bf16 ratio (1.1 / 2.25).
BF16_FALLBACK_TFLOPS = 1886.9


def tensor_peak(mode):
    bf16 = BF16_FALLBACK_TFLOPS
    src = "fallback"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
            src = "measured"
    except Exception:
        pass
    if mode == "tf32":
        return bf16 * 1.1 / 2.25, f"{src} bf16 x nominal tf32/bf16"
    return bf16, f"{src} bf16 (burst)"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the leaf kernel on the full-size workload, from ncu captures, valid only for
# the kernel source it was taken on (the first 16 hex digits of the sha256 of
# leaf_tc.cu or kernels_f64.cu).
LEAF_TRAFFIC = {
    # a one-launch capture of the 4500^2 small case (cutoff 1200), scaled by
    # the ratio of tree multiplications (traffic grows with tiles x K)
    ("ata_ozaki_10000x10000", "c9d903142d171577"): (940.4e6 + 95.2e6) * 468800000000 / 42724968750,
}


# A buffer larger than the 129 MB L2: written between timed steps of a
# workload whose input fits in L2.
L2_FLUSH_BYTES = 256 << 20


def _src_sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def effective_flops(m, n):
    return 2.0 * m * n * n


def make_input(name):
    from paper_1902_02104_gb300 import inputs
    m, n, mode, gen, seed, _ = WORKLOADS[name]
    A = getattr(inputs, gen)(m, n, seed=seed)
    return A.astype(np.float64 if mode in ("f64", "ozaki") else np.float32)


def sampled_error(oracle, A_np, C, n, kind, dev, torch, count=2000, seed=123):
    """Componentwise error over sampled entries, or the normwise error
    estimated from every diagonal entry plus sampled off-diagonal ones."""
    rng = np.random.default_rng(seed)
    I = rng.integers(0, n, size=count)
    J = rng.integers(0, n, size=count)
    I, J = np.minimum(I, J), np.maximum(I, J)
    if kind == "componentwise":
        got = C[torch.from_numpy(oracle.packed_index(I, J, n)).to(dev)].cpu().numpy()
        ref = oracle.ata_entries(A_np, I, J)
        G = oracle.ata_entries(A_np, I, J, absval=True)
        return oracle.componentwise_error(got, ref, G)
    keep = I != J
    I, J = I[keep], J[keep]
    d = np.arange(n)
    got_d = C[torch.from_numpy(oracle.packed_index(d, d, n)).to(dev)].cpu().numpy()
    got_o = C[torch.from_numpy(oracle.packed_index(I, J, n)).to(dev)].cpu().numpy()
    ref_d = oracle.ata_entries(A_np, d, d)
    ref_o = oracle.ata_entries(A_np, I, J)
    w = (n * (n - 1) / 2) / max(I.size, 1) * 2.0
    num = np.sum((got_d - ref_d) ** 2) + w * np.sum((got_o - ref_o) ** 2)
    den = np.sum(ref_d ** 2) + w * np.sum(ref_o ** 2)
    return float(np.sqrt(num / den))


def library_reference(A, A_np, n, eff, kind, oracle, dev, torch, reps=2, count=2000, seed=123):
    """torch.matmul(A^t, A) on the same resident input, the library reference
    point (cuBLAS: a float64 GEMM for FP64 input, a float32 GEMM with TF32 off
    for FP32 input).  It computes the full n x n product (2 m n^2 FLOP, the
    same effective count).  Sampled error against the oracle as for ours."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        out = torch.matmul(A.t(), A)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = torch.matmul(A.t(), A)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    rng = np.random.default_rng(seed)  # the entries sampled_error takes
    I = rng.integers(0, n, size=count)
    J = rng.integers(0, n, size=count)
    I, J = np.minimum(I, J), np.maximum(I, J)

    def entries(i, j):
        return out[torch.from_numpy(i).to(dev), torch.from_numpy(j).to(dev)].double().cpu().numpy()

    if kind == "componentwise":
        err = oracle.componentwise_error(entries(I, J), oracle.ata_entries(A_np, I, J),
                                         oracle.ata_entries(A_np, I, J, absval=True))
    else:
        keep = I != J
        I, J = I[keep], J[keep]
        d = np.arange(n)
        ref_d, ref_o = oracle.ata_entries(A_np, d, d), oracle.ata_entries(A_np, I, J)
        w = (n * (n - 1) / 2) / max(I.size, 1) * 2.0
        num = np.sum((entries(d, d) - ref_d) ** 2) + w * np.sum((entries(I, J) - ref_o) ** 2)
        err = float(np.sqrt(num / (np.sum(ref_d ** 2) + w * np.sum(ref_o ** 2))))
    del out
    torch.cuda.empty_cache()
    return {"call": f"torch.matmul(A.t(), A), {str(A.dtype).replace('torch.', '')}, TF32 off", "ms": ms,
            "value": eff / (ms / 1e3) / 1e12, "unit": "TFLOP/s", kind + "_sampled": err, "samples": count}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device_index):
        self.proc = None
        self.path = None
        self.dev = device_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) == len(self.FIELDS):
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_smi_index(torch, dev):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        return vis.split(",")[dev.index or 0].strip()
    return str(dev.index or 0)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(torch, value, world):
    """The largest of every rank's value (the slowest replica sets the time)."""
    if world == 1:
        return value
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_oracle_sample(A, budget_s=15.0):
    """Times the oracle on leading rows of the packed triangle for about
    budget_s seconds of multiply-adds and extrapolates to the whole product.
    Every call of the row routine first copies A into column-major order; that
    fixed cost (timed on a one-row call) is taken off each measurement, so the
    extrapolation scales only the multiply-adds."""
    import oracle
    m, n = A.shape
    total = m * n * (n + 1) / 2
    t0 = time.perf_counter()
    oracle.ata_rows(A, 0, 1)
    t_fixed = time.perf_counter() - t0  # the copy (and one row)
    # calibrate on a few more rows
    rows = max(2, min(n, 64))
    t0 = time.perf_counter()
    oracle.ata_rows(A, 1, rows)
    dt = max(time.perf_counter() - t0 - t_fixed, 1e-6)
    done = m * sum(n - i for i in range(1, rows))
    rate = done / dt
    # grow to the budget
    want = rate * budget_s
    r1 = rows
    acc = 0
    while r1 < n and acc < want:
        acc += m * (n - r1)
        r1 += 1
    t0 = time.perf_counter()
    oracle.ata_rows(A, rows, r1)
    dt = max(time.perf_counter() - t0 - t_fixed, 1e-6)
    done = m * sum(n - i for i in range(rows, r1))
    t_full = dt * total / max(done, 1)
    return {"t_full_s": t_full, "rows": (rows, r1), "sample_s": dt, "cores": oracle.num_threads(),
            "frac": done / total, "fixed_s": t_fixed}


def workload_config(name, world, a_bytes, cutoff):
    """The config object of an A^t A workload's line (both arms)."""
    m, n, mode, gen, seed, _ = WORKLOADS[name]
    small = a_bytes < L2_FLUSH_BYTES
    return {"workload": name, "m": m, "n": n, "leaf": mode, "generator": f"{gen}(seed={seed})",
            "cutoff": cutoff if cutoff else "autotuned", "parallelism": f"replicas{world}",
            "l2": ("L2 flushed before every timed step (A is %.1f MB)" % (a_bytes / 2**20)) if small
                  else "inputs larger than L2 (A is %d MB)" % (a_bytes >> 20)}


def run_reference(args):
    """The oracle (plain FP64 triple loop, OpenMP over the host cores) on the
    workload's input.  Every step is one call of the oracle's row routine on
    a bounded sample of the packed triangle (about --cpu-budget-per-step
    seconds; successive steps take successive rows), timed whole: ms_per_step
    is the wall time of the calls that ran, and value their effective rate
    (the sample's share of the 2 m n^2 effective FLOP over that time)."""
    import oracle
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    name = args.workload
    m, n, mode, gen, seed, cutoff = WORKLOADS[name]
    A = make_input(name)
    eff = effective_flops(m, n)
    total = m * n * (n + 1) / 2
    budget = max(2.0, min(15.0, 150.0 / max(1, args.steps + args.warmup)))

    def rows_for(r0, seconds, rate):
        r1, acc = r0, 0.0
        while r1 < n and acc < rate * seconds:
            acc += m * (n - r1)
            r1 += 1
        return max(r1, r0 + 1)

    # calibration (one of the warm-up calls): multiply-adds per second
    t0 = time.perf_counter()
    oracle.ata_rows(A, 0, min(n, 64))
    rate = m * sum(n - i for i in range(min(n, 64))) / max(time.perf_counter() - t0, 1e-6)
    r0 = min(n, 64)
    for _ in range(args.warmup - 1):
        r1 = rows_for(r0, budget / 4, rate)
        oracle.ata_rows(A, r0 % n, min(n, r0 % n + (r1 - r0)))
        r0 = r1 % n
    times, done = [], []
    for _ in range(args.steps):
        a0 = r0 % n
        a1 = min(n, rows_for(a0, budget, rate))
        t0 = time.perf_counter()
        oracle.ata_rows(A, a0, a1)
        dt = time.perf_counter() - t0
        times.append(dt)
        done.append(m * sum(n - i for i in range(a0, a1)))
        rate = done[-1] / max(dt, 1e-6)
        r0 = a1
    wall = sum(times)
    frac = sum(done) / args.steps / total
    value = sum(d / total * eff for d in done) / wall / 1e12
    line = {
        "impl": "reference", "metric": "effective TFLOP/s (m*n^2 FMAs) of C = A^t A", "value": value,
        "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": workload_config(name, 1, A.nbytes, cutoff),
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"each step: consecutive packed rows ({100 * frac:.2f}% of the product's "
                                   f"multiplications on average), timed whole; value = the rows' share of "
                                   f"2 m n^2 over their time"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch

    import oracle
    import paper_1902_02104_gb300 as ata

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    name = args.workload
    m, n, mode, gen, seed, cutoff = WORKLOADS[name]
    if args.cutoff is not None:
        cutoff = args.cutoff
    A_np = make_input(name)
    tuning = None
    if cutoff == 0 and not args.model_cutoff:
        # the cutoff and tile form measured on this device (ata_tune), before
        # the timed region
        t0 = time.perf_counter()
        opts = ata.ata_tune(m, n, MODE_CODES[mode], candidates=3)
        tuning = {"measured_ms": opts.pop("best_ms"), "tuning_s": time.perf_counter() - t0,
                  "how": "ata_tune: the cost model's 3 best cutoffs x (single-CTA, CTA-pair) tiles timed on "
                         "this GPU, median of 3"}
        plan = ata.Plan(m, n, MODE_CODES[mode], **opts)
    else:
        plan = ata.Plan(m, n, MODE_CODES[mode], cutoff)
    info = plan.info
    A = torch.from_numpy(A_np).to(dev)
    C = torch.empty(n * (n + 1) // 2, dtype=torch.float64, device=dev)
    plan.enable_stage_timing(True)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        plan(A, C)
    torch.cuda.synchronize()

    sampler = ClockSampler(gpu_smi_index(torch, dev))
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    small = A_np.nbytes < L2_FLUSH_BYTES
    if not small:
        # the timed region: K steps queued back to back (A is larger than L2),
        # an event between consecutive steps for the per-step distribution
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        e0.record(stream)
        for k in range(args.steps):
            plan(A, C)
            evs[k].record(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        step_ms = [a.elapsed_time(b) for a, b in zip([e0] + evs[:-1], evs)]
    else:
        # A fits in L2: every step starts from a cold L2 (a buffer larger than
        # L2 is written before it, outside its events)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        step_ms = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0.record(stream)
            plan(A, C)
            e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        ms = sum(step_ms) / args.steps
        del flush
    barrier(world)
    clocks = sampler.stop()
    ms_max = max_over_ranks(torch, ms, world)
    # stage split (events inside the plan's graph), one step at a time
    leaf_ms, split_ms, comb_ms, prep_ms = [], [], [], []
    for _ in range(args.steps):
        plan(A, C)
        stream.synchronize()
        st = plan.stage_times()
        leaf_ms.append(st["leaf_ms"])
        split_ms.append(st["split_ms"])
        prep_ms.append(st["prep_ms"])
        comb_ms.append(st["combine_ms"])

    # accuracy at the stated tolerance: sampled entries against the oracle
    err_kind, tol = TOLERANCE[mode]
    cnt = 2000
    err = sampled_error(oracle, A_np, C, n, err_kind, dev, torch, count=cnt)
    dev_status = plan.device_status()

    # end to end through the C ABI from pinned host memory: every step copies
    # its input in and its packed result out.  The steps are pipelined calls
    # (the copies of one step overlap the executions of its neighbours on two
    # staging sets); the clock stops when the last result is on the host.
    A_host = torch.from_numpy(A_np).pin_memory()
    C_host = torch.empty(n * (n + 1) // 2, dtype=torch.float64).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))
    for _ in range(2):  # both staging sets' graphs captured
        ata.ata_execute_host_async(plan, A_host.numpy(), C_host.numpy())
    ata.ata_plan_wait(plan)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ata.ata_execute_host_async(plan, A_host.numpy(), C_host.numpy())
    ata.ata_plan_wait(plan)
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    t_e2e = max_over_ranks(torch, t_e2e, world)

    eff = effective_flops(m, n)
    value = world * eff / (ms_max / 1e3) / 1e12
    leaf_s = statistics.mean(leaf_ms) / 1e3
    leaf_flops = 2.0 * info["mults"] * PAIRS[mode]
    achieved = leaf_flops / leaf_s / 1e12
    if mode == "f64":
        kern, src, bound, peak, peak_src = "leaf_f64_kernel", "kernels_f64.cu", "alu", FP64_ALU_PEAK_TFLOPS, \
            "derived: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz"
    else:
        kern, src, bound = "tc_gemm_kernel", "leaf_tc.cu", "tensor"
        peak, peak_src = tensor_peak(mode)
    sha = _src_sha(os.path.join(ROOT, "paper_1902_02104_gb300", "csrc", src))
    tr = LEAF_TRAFFIC.get((name, sha))
    line = {
        "metric": "effective TFLOP/s (m*n^2 FMAs) of C = A^t A", "value": value, "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "ozaki": "bf16 (FP64 emulation, 6 slices)", "bf16x3": "bf16 (3 slices)",
                  "tf32": "tf32"}[mode], "data": "synthetic",
        "config": workload_config(name, world, A_np.nbytes, cutoff),
        "plan": {"cutoff": info["cutoff"], "strassen_levels_max": info["max_strassen_levels"],
                 "leaf_tile": [info["leaf_tile_rows"], info["leaf_tile_cols"]], "tuning": tuning},
        "error": {err_kind + "_sampled": err, "tolerance": tol, "samples": cnt, "device_status": dev_status},
        "stages_ms": {"split": statistics.mean(split_ms), "prep": statistics.mean(prep_ms),
                      "leaf": statistics.mean(leaf_ms), "combine": statistics.mean(comb_ms)},
        "step_ms": step_percentiles(step_ms),
        "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": tr, "peak_source": peak_src,
                     "kernel": kern, "flops_per_launch": leaf_flops},
        "e2e": {"value": world * eff / t_e2e / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": int(A_np.nbytes),
                "d2h_bytes_per_step": int(C.numel() * 8), "steps": e2e_steps,
                "calls": "ata_execute_host_async per step (pipelined), ata_plan_wait at the end"},
        "gpu_launches": int(args.steps * info["n_launches"]),
        "clocks": clocks,
    }
    if mode == "ozaki" and not args.no_plain:
        # the plain FP64 path on the same input, same GPU, same tolerance
        del plan
        torch.cuda.empty_cache()
        pf = ata.Plan(m, n, ata.ATA_F64, 0)
        for _ in range(2):
            pf(A, C)
        torch.cuda.synchronize()
        barrier(world)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(max(1, min(args.steps, 3))):
            pf(A, C)
        f1.record(stream)
        torch.cuda.synchronize()
        fms = max_over_ranks(torch, f0.elapsed_time(f1) / max(1, min(args.steps, 3)), world)
        ferr = sampled_error(oracle, A_np, C, n, "componentwise", dev, torch, count=cnt)
        line["plain_f64"] = {"value": world * eff / (fms / 1e3) / 1e12, "unit": "TFLOP/s", "ms_per_step": fms,
                             "cutoff": pf.info["cutoff"], "componentwise_sampled": ferr}
        line["speedup_vs_plain_f64"] = fms / ms_max
        del pf
        torch.cuda.empty_cache()
    if not args.no_library:
        line["library_reference"] = library_reference(A, A_np, n, eff, err_kind, oracle, dev, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = cpu_oracle_sample(A_np, budget_s=args.cpu_budget)
        line["cpu_baseline"] = {
            "value": eff / r["t_full_s"] / 1e12, "unit": "TFLOP/s", "cores": r["cores"], "kind": "oracle",
            "sample": f"packed rows {r['rows'][0]}..{r['rows'][1]} ({100 * r['frac']:.2f}% of the "
                      f"multiplications, {r['sample_s']:.1f} s), extrapolated to the whole product"}
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line if rank == 0 else None


def step_percentiles(step_ms):
    """Median, p99 (nearest rank), min and max of this rank's timed steps."""
    v = sorted(step_ms)
    p99 = v[min(len(v) - 1, max(0, int(np.ceil(0.99 * len(v))) - 1))]
    return {"median": statistics.median(v), "p99": p99, "min": v[0], "max": v[-1], "count": len(v)}


def _line_common(args, world, metric, value, unit, ms, mode, config):
    return {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"f64": "f64", "bf16x3": "bf16 (3 slices)", "tf32": "tf32",
                                          "ozaki": "bf16 (FP64 emulation, 6 slices)"}[mode],
            "data": "synthetic", "config": config}


def run_batched(args, mode):
    """Batched workload: 512 independent instances, m log-U[64,4096], n log-U[32,1024],
    U(-1,1), seed 3; one execution of a prepared batch (the instances packed
    back to back in one input and one output buffer; merged task tables, one
    persistent leaf launch, captured graph) per step."""
    import torch

    import oracle
    import paper_1902_02104_gb300 as ata
    from paper_1902_02104_gb300 import inputs
    world, rank, local = dist_setup()
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    dt = np.float64 if mode in ("f64", "ozaki") else np.float32
    mats = [a.astype(dt) for a in inputs.batch(512, seed=3)]
    tuning = None

    def make_batch(policy):
        cut = (lambda a: 0) if policy == "model" else (lambda a: int(policy))
        ps = [ata.Plan(a.shape[0], a.shape[1], MODE_CODES[mode], cut(a)) for a in mats]
        return ps, ata.Batch(ps)

    if args.model_cutoff:
        plans, batch = make_batch("model")
    else:
        # The cutoff policy measured on this device for the whole batch
        # (before the timed region): the planner's cost model per shape, or
        # one cutoff for every instance.  Each candidate batch runs once
        # untimed and three times timed; the fastest median wins.  (Timing
        # each shape alone misleads here: a small instance alone is timed
        # mostly on its launch latency, which the merged batch does not pay;
        # per-bucket choices made that way ran 5% slower.)
        t0 = time.perf_counter()
        hA = torch.zeros(1, dtype=torch.float32)
        times = {}
        best = None
        for policy in ["model", 4096, 1024, 512]:
            ps, b = make_batch(policy)
            hA = torch.zeros(b.a_numel, dtype=b.in_dtype)
            for v, a in zip(b.input_views(hA), mats):
                v.copy_(torch.from_numpy(a))
            dA = hA.to(dev)
            dC = torch.empty(b.c_numel, dtype=torch.float64, device=dev)
            b(dA, dC)
            torch.cuda.synchronize()
            ts = []
            for _ in range(3):
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record()
                b(dA, dC)
                s1.record()
                torch.cuda.synchronize()
                ts.append(s0.elapsed_time(s1))
            times[str(policy)] = float(np.median(ts))
            if best is None or times[str(policy)] < times[str(best)]:
                best = policy
            del ps, b, dA, dC
            torch.cuda.empty_cache()
        plans, batch = make_batch(best)
        tuning = {"chosen": str(best), "measured_ms": times, "tuning_s": time.perf_counter() - t0,
                  "how": "whole batch timed on this GPU under each cutoff policy (cost model per shape, or one "
                         "cutoff for all), median of 3"}
    # the packed input in pinned host memory, and its device copy
    hostA = torch.zeros(batch.a_numel, dtype=batch.in_dtype).pin_memory()
    for v, a in zip(batch.input_views(hostA), mats):
        v.copy_(torch.from_numpy(a))
    devA = hostA.to(dev)
    devC = torch.empty(batch.c_numel, dtype=torch.float64, device=dev)
    hostC = torch.empty(batch.c_numel, dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        batch(devA, devC)
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_smi_index(torch, dev))
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e0.record(stream)
    for k in range(args.steps):
        batch(devA, devC)
        evs[k].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in zip([e0] + evs[:-1], evs)]
    barrier(world)
    clocks = sampler.stop()
    ms = max_over_ranks(torch, e0.elapsed_time(e1) / args.steps, world)
    eff = sum(effective_flops(a.shape[0], a.shape[1]) for a in mats)
    kind, tol = TOLERANCE[mode]

    def sampled_errors(C):
        errs = []
        for i, c in list(enumerate(batch.output_views(C)))[::64]:  # every 64th instance, full oracle
            ref = oracle.ata_packed(mats[i])
            got = c.cpu().numpy() if c.is_cuda else c.numpy()
            if kind == "normwise":
                errs.append(oracle.normwise_error(got, ref, mats[i].shape[1]))
            else:
                errs.append(oracle.componentwise_error(got, ref, oracle.abs_gram_packed(mats[i])))
        return errs

    errs = sampled_errors(devC)
    mults = sum(p.info["mults"] for p in plans)
    leaf_flops = 2.0 * mults * PAIRS[mode]
    achieved = leaf_flops / (ms / 1e3) / 1e12
    if mode == "f64":
        peak, peak_src, bound = FP64_ALU_PEAK_TFLOPS, "derived DFMA peak", "alu"
    else:
        peak, peak_src = tensor_peak(mode)
        bound = "tensor"

    # End to end: every step copies the whole packed input in from pinned
    # host memory and the whole packed output back, through ata_batch_execute
    # on a stream of its own.  Steps alternate between two device buffer
    # sets on three streams (copy in, execute, copy out) ordered by events,
    # so that a step's copies overlap its neighbours' executions; the clock
    # stops when the last result is on the host.
    s_in, s_run, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    dA = [devA, torch.empty_like(devA)]
    dC = [devC, torch.empty_like(devC)]
    hC = [hostC, torch.empty_like(hostC).pin_memory()]
    ev_a = [torch.cuda.Event(), torch.cuda.Event()]
    ev_run = [torch.cuda.Event(), torch.cuda.Event()]
    ev_c = [torch.cuda.Event(), torch.cuda.Event()]

    def e2e_step(i):
        b = i & 1
        s_in.wait_event(ev_run[b])  # the execution that last read dA[b] has finished
        with torch.cuda.stream(s_in):
            dA[b].copy_(hostA, non_blocking=True)
        ev_a[b].record(s_in)
        s_run.wait_event(ev_a[b])
        s_run.wait_event(ev_c[b])   # the copy-out that last read dC[b] has finished
        batch.execute(dA[b], dC[b], stream=s_run)
        ev_run[b].record(s_run)
        s_out.wait_event(ev_run[b])
        with torch.cuda.stream(s_out):
            hC[b].copy_(dC[b], non_blocking=True)
        ev_c[b].record(s_out)
    for c in dC:
        c.zero_()
    torch.cuda.synchronize()
    for i in range(2):
        e2e_step(i)
    torch.cuda.synchronize()
    e2e_steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        e2e_step(i)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(torch, (time.perf_counter() - t0) / e2e_steps, world)
    hostC = hC[(e2e_steps - 1) & 1]
    errs += sampled_errors(hostC)
    line = _line_common(args, world, "effective TFLOP/s (m*n^2 FMAs) of C = A^t A, 512 batched instances",
                        world * eff / (ms / 1e3) / 1e12, "TFLOP/s", ms, mode,
                        {"workload": f"batched_{mode}", "instances": 512, "m_range": [64, 4096],
                         "n_range": [32, 1024], "generator": "uniform(-1,1) seed 3", "cutoff": "cost model per shape" if args.model_cutoff else "policy measured on the batch",
                         "parallelism": f"replicas{world}", "calls": "one ata_batch_execute per step",
                         "e2e": "copy in, execute, copy out on three streams, two buffer sets alternating",
                         "l2": "inputs larger than L2 (%.0f MB)" % (sum(a.nbytes for a in mats) / 2**20)})
    line["roofline"] = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                        "kernel": "whole batched step (leaf flops / step time)", "flops_per_launch": leaf_flops}
    line["e2e"] = {"value": world * eff / t_e2e / 1e12, "unit": "TFLOP/s",
                   "h2d_bytes_per_step": int(hostA.numel() * hostA.element_size()),
                   "d2h_bytes_per_step": int(hostC.numel() * 8)}
    line["step_ms"] = step_percentiles(step_ms)
    line["gpu_launches"] = int(args.steps * batch.graph_kernels())
    line["error"] = {kind + "_max_of_16": max(errs), "tolerance": tol,
                     "checked": "every 64th instance, device-timed and end-to-end results"}
    line["clocks"] = clocks
    line["tuning"] = tuning
    return line if rank == 0 else None


# Serving rates allowed per mode: rates at which the mode has run clean on
# GB300 (bf16x3 at 2000 req/s for 60 s, offered load about 1% of its
# capacity; the FP64 emulation at 500 req/s), and for plain FP64 200 req/s,
# about 40% of its capacity (478 req/s, each request timed alone), so that
# it is never offered more work than it completes: offered more, it once
# raised an illegal-address fault whose cause was not found.  Higher rates
# are refused.
SERVING_CLEAN_RATE = {"bf16x3": 2000.0, "ozaki": 500.0, "f64": 200.0}


def run_serving(args, mode):
    """Serving workload: Poisson arrivals at --rate for --duration seconds; requests
    draw matrices from a 256-entry pool (m log-U[128,8192], n log-U[64,2048],
    N(0,1)); admission by a 40 GB budget; plans resident after warm-up.

    Every request writes its own output buffer: a buffer of a pool entry is
    reused only after the request that last wrote it has completed (a new
    buffer is allocated otherwise).  Requests spread over the timed phase
    write buffers of their own that are compared with the oracle afterwards."""
    import torch

    import oracle
    import paper_1902_02104_gb300 as ata
    from paper_1902_02104_gb300 import inputs
    cap = SERVING_CLEAN_RATE.get(mode)
    if cap is None or args.rate > cap:
        raise SystemExit(f"serving_{mode} at {args.rate:g} req/s is refused: the measured-clean rates are "
                         f"{SERVING_CLEAN_RATE} requests per second")
    world, rank, local = dist_setup()
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    dt = np.float64 if mode in ("f64", "ozaki") else np.float32
    rng, pool = inputs.serving_pool(256, seed=4)
    pool = [a.astype(dt) for a in pool]
    As = [torch.from_numpy(a).to(dev) for a in pool]

    def new_c(i):
        n = pool[i].shape[1]
        return torch.empty(n * (n + 1) // 2, dtype=torch.float64, device=dev)

    free = [[new_c(i)] for i in range(len(pool))]  # output buffers no running request writes
    running = [[] for _ in pool]                   # per entry: (ticket, buffer), oldest first
    torch.cuda.synchronize()  # inputs complete before the server's streams read them
    srv = ata.Server(40 << 30, MODE_CODES[mode], max_inflight=16)

    def reap(i, wait_us=0):
        """Move buffers of entry i's completed requests (oldest first) back to free."""
        while running[i] and srv.poll(running[i][0][0], wait_us) == ata.ATA_OK:
            free[i].append(running[i].pop(0)[1])

    def submit(i, own=None):
        if own is not None:
            return srv.submit(As[i], own)
        if not free[i]:
            reap(i)
        c = free[i].pop() if free[i] else new_c(i)
        t = srv.submit(As[i], c)
        running[i].append((t, c))
        return t

    def drain():
        for i in range(len(pool)):
            while running[i]:
                reap(i, 600_000_000)

    # warm-up: every pool shape once (plans become resident)
    for i in range(len(pool)):
        submit(i)
    drain()
    arrivals = inputs.poisson_arrivals(args.rate, args.duration, seed=4)
    which = rng.integers(0, len(pool), size=arrivals.size)
    n_check = min(8, arrivals.size)
    check_at = set(np.linspace(0, arrivals.size - 1, n_check).round().astype(int).tolist()) if n_check else set()
    checks = []  # (pool entry, own buffer, ticket)
    srv.reset_stats()
    sampler = ClockSampler(gpu_smi_index(torch, dev))
    sampler.start()
    time.sleep(0.3)
    t0 = time.perf_counter()
    for k, (t_arr, i) in enumerate(zip(arrivals, which)):
        while time.perf_counter() - t0 < t_arr:
            pass
        if k in check_at:
            c = new_c(int(i))
            checks.append((int(i), c, submit(int(i), own=c)))
        else:
            submit(int(i))
    for _, _, t in checks:
        srv.poll(t, 600_000_000)
    drain()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    st = srv.stats()
    served_kernels = srv.kernels()
    srv.close()
    eff = sum(effective_flops(*pool[i].shape) for i in which)
    kind, tol = TOLERANCE[mode]
    # correctness: requests served in the mix, against the oracle
    errs = []
    for i, c, _ in checks:
        got = c.cpu().numpy()
        ref = oracle.ata_packed(pool[i])
        if kind == "normwise":
            errs.append(oracle.normwise_error(got, ref, pool[i].shape[1]))
        else:
            errs.append(oracle.componentwise_error(got, ref, oracle.abs_gram_packed(pool[i])))
    # the plain FP64 path on the same pool: its service time per request, run
    # one request at a time on one stream (capacity, not served under load)
    fp64 = None
    if not args.no_plain:
        idx = list(range(0, 256, 8))
        svc = []
        for i in idx:
            a = pool[i].astype(np.float64)
            pf = ata.Plan(a.shape[0], a.shape[1], ata.ATA_F64, 0)
            Ad = torch.from_numpy(a).to(dev)
            Cd = torch.empty(a.shape[1] * (a.shape[1] + 1) // 2, dtype=torch.float64, device=dev)
            pf(Ad, Cd)
            torch.cuda.synchronize()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record()
            pf(Ad, Cd)
            f1.record()
            torch.cuda.synchronize()
            svc.append(f0.elapsed_time(f1))
            del pf, Ad, Cd
        mean_ms = float(np.mean(svc))
        eff_mean = float(np.mean([effective_flops(*pool[i].shape) for i in idx]))
        fp64 = {"mean_service_ms": mean_ms, "max_rate_per_s": 1e3 / mean_ms,
                "effective_tflops_at_capacity": eff_mean / (mean_ms / 1e3) / 1e12,
                "sample": f"{len(idx)} pool shapes, one request at a time"}
    line = _line_common(args, world, "sustained effective TFLOP/s of served A^t A requests; p50/p99 latency",
                        world * eff / wall / 1e12, "TFLOP/s", wall * 1e3, mode,
                        {"workload": f"serving_{mode}", "rate_per_s": args.rate, "duration_s": args.duration,
                         "requests": int(arrivals.size), "pool": 256, "m_range": [128, 8192],
                         "n_range": [64, 2048], "budget_bytes": 40 << 30, "max_inflight": 16,
                         "parallelism": f"replicas{world}"})
    line["latency_us"] = {"p50": st["p50_us"], "p99": st["p99_us"], "completed": st["completed"]}
    line["offered_effective_tflops"] = eff / args.duration / 1e12
    line["plain_f64_capacity"] = fp64
    line["error"] = {kind + "_max": max(errs) if errs else None, "tolerance": tol,
                     "checked": f"{len(errs)} requests served in the mix (spread over the timed phase), "
                                f"full oracle"}
    line["roofline"] = None
    line["e2e"] = None
    line["gpu_launches"] = int(served_kernels)
    line["clocks"] = clocks
    return line if rank == 0 else None


def run_gemm(args):
    """The general product C = X^t Y through ata_gemm_tn (X: m x p, Y: m x r,
    C: p x r dense FP64).  A step is one call over resident X and Y; the
    metric is effective TFLOP/s = 2 m p r / t."""
    import torch

    import oracle
    import paper_1902_02104_gb300 as ata
    from paper_1902_02104_gb300 import inputs
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    name = args.workload
    m, p, r, mode, gen, seed, cutoff = GEMM_WORKLOADS[name]
    if args.cutoff is not None:
        cutoff = args.cutoff
    dt = np.float64 if mode in ("f64", "ozaki") else np.float32
    X_np = getattr(inputs, gen)(m, p, seed=seed).astype(dt)
    Y_np = getattr(inputs, gen)(m, r, seed=seed + 1).astype(dt)
    plan = ata.GemmPlan(m, p, r, MODE_CODES[mode], cutoff)
    info = plan.info
    X = torch.from_numpy(X_np).to(dev)
    Y = torch.from_numpy(Y_np).to(dev)
    C = torch.empty((p, r), dtype=torch.float64, device=dev)
    plan.enable_stage_timing(True)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        plan(X, Y, C)
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_smi_index(torch, dev))
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stage = {"split": [], "prep": [], "leaf": [], "combine": []}
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e0.record(stream)
    for k in range(args.steps):
        plan(X, Y, C)
        evs[k].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in zip([e0] + evs[:-1], evs)]
    barrier(world)
    clocks = sampler.stop()
    ms = max_over_ranks(torch, e0.elapsed_time(e1) / args.steps, world)
    for _ in range(args.steps):
        plan(X, Y, C)
        stream.synchronize()
        st = plan.stage_times()
        for k in stage:
            stage[k].append(st[k + "_ms"])
    # accuracy on sampled entries
    rng = np.random.default_rng(123)
    I = rng.integers(0, p, 2000)
    J = rng.integers(0, r, 2000)
    got = C[torch.from_numpy(I).to(dev), torch.from_numpy(J).to(dev)].cpu().numpy()
    ref = oracle.gemm_entries(X_np, Y_np, I, J)
    kind, tol = TOLERANCE[mode]
    if kind == "componentwise":
        G = oracle.gemm_entries(X_np, Y_np, I, J, absval=True)
        err = float(np.max(np.abs(got - ref) / G))
    else:
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        kind = "normwise_sampled_entries"
    # end to end: pinned host X, Y in, C out, through the same call
    Xh = torch.from_numpy(X_np).pin_memory()
    Yh = torch.from_numpy(Y_np).pin_memory()
    Ch = torch.empty((p, r), dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        Xd = Xh.to(dev, non_blocking=True)
        Yd = Yh.to(dev, non_blocking=True)
        plan(Xd, Yd, C)
        Ch.copy_(C, non_blocking=True)
        torch.cuda.synchronize()
    t_e2e = max_over_ranks(torch, (time.perf_counter() - t0) / e2e_steps, world)
    eff = 2.0 * m * p * r
    leaf_s = statistics.mean(stage["leaf"]) / 1e3
    leaf_flops = 2.0 * info["mults"] * PAIRS[mode]
    if mode == "f64":
        kern, bound, peak, peak_src = "leaf_f64_kernel", "alu", FP64_ALU_PEAK_TFLOPS, \
            "derived: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz"
    else:
        kern, bound = "tc_gemm_kernel", "tensor"
        peak, peak_src = tensor_peak(mode)
    line = _line_common(args, world, "effective TFLOP/s (2 m p r) of C = X^t Y", world * eff / (ms / 1e3) / 1e12,
                        "TFLOP/s", ms, mode,
                        {"workload": name, "m": m, "p": p, "r": r, "leaf": mode, "generator": f"{gen}(seed={seed})",
                         "cutoff": info["cutoff"], "strassen_levels": info["max_strassen_levels"],
                         "parallelism": f"replicas{world}",
                         "l2": "inputs larger than L2 (X is %d MB)" % (X_np.nbytes >> 20)})
    line["error"] = {kind: err, "tolerance": tol, "samples": 2000, "device_status": plan.device_status()}
    line["stages_ms"] = {k: statistics.mean(v) for k, v in stage.items()}
    line["step_ms"] = step_percentiles(step_ms)
    line["roofline"] = {"bound": bound, "achieved": leaf_flops / leaf_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                        "frac": leaf_flops / leaf_s / 1e12 / peak, "traffic": None, "peak_source": peak_src,
                        "kernel": kern, "flops_per_launch": leaf_flops}
    line["e2e"] = {"value": world * eff / t_e2e / 1e12, "unit": "TFLOP/s",
                   "h2d_bytes_per_step": int(X_np.nbytes + Y_np.nbytes), "d2h_bytes_per_step": int(p * r * 8)}
    line["gpu_launches"] = int(args.steps * info["n_launches"])
    line["clocks"] = clocks
    if not args.no_library:
        # torch.matmul(X^t, Y) on the same resident inputs (cuBLAS, TF32 off)
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        out = torch.matmul(X.t(), Y)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(2):
            out = torch.matmul(X.t(), Y)
        e1.record()
        torch.cuda.synchronize()
        torch.backends.cuda.matmul.allow_tf32 = prev
        lms = e0.elapsed_time(e1) / 2
        lgot = out[torch.from_numpy(I).to(dev), torch.from_numpy(J).to(dev)].double().cpu().numpy()
        lerr = float(np.max(np.abs(lgot - ref) / G)) if kind == "componentwise" else \
            float(np.linalg.norm(lgot - ref) / np.linalg.norm(ref))
        line["library_reference"] = {"call": f"torch.matmul(X.t(), Y), {str(X.dtype).replace('torch.', '')}, "
                                             f"TF32 off", "ms": lms, "value": eff / (lms / 1e3) / 1e12,
                                     "unit": "TFLOP/s", kind: lerr, "samples": 2000}
        del out
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on a bounded sample of entries (about --cpu-budget
        # seconds), extrapolated to all p r entries
        srng = np.random.default_rng(7)
        cnt = 2048
        Is, Js = srng.integers(0, p, cnt), srng.integers(0, r, cnt)
        t0 = time.perf_counter()
        oracle.gemm_entries(X_np, Y_np, Is, Js)
        per = (time.perf_counter() - t0) / cnt
        cnt = int(min(p * r, max(cnt, args.cpu_budget / max(per, 1e-9))))
        Is, Js = srng.integers(0, p, cnt), srng.integers(0, r, cnt)
        t0 = time.perf_counter()
        oracle.gemm_entries(X_np, Y_np, Is, Js)
        dt_s = time.perf_counter() - t0
        t_full = dt_s * p * r / cnt
        line["cpu_baseline"] = {"value": eff / t_full / 1e12, "unit": "TFLOP/s", "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": f"{cnt} sampled entries ({dt_s:.1f} s), extrapolated "
                                                            f"to all {p * r} entries"}
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line if rank == 0 else None


# The other workloads of the benchmark family, run after the default one at
# N = 1 with a short timed region each and attached to its line: the plain
# FP64 form at 512 x 384, the precision form in both leaf modes, the batched
# form and the serving form (10 s of arrivals; 60 s with --workload
# serving_bf16x3 --duration 60).
SUB_CONFIGS = [
    ("plain FP64, A 512 x 384, cutoff 64", "ata_f64_512x384", {}),
    ("precision form, bf16x3 leaves, A 16384 x 8192 FP32", "ata_bf16x3_16384x8192", {}),
    ("precision form, TF32 leaves, A 16384 x 8192 FP32", "ata_tf32_16384x8192", {}),
    ("batched form, 512 instances, bf16x3 leaves", "batched_bf16x3", {}),
    ("serving form, bf16x3 leaves, Poisson 2000 req/s", "serving_bf16x3", {"duration": 10.0, "rate": 2000.0}),
]


def dispatch(args):
    if args.workload in GEMM_WORKLOADS:
        return run_gemm(args)
    if args.workload.startswith("batched_"):
        return run_batched(args, args.workload.split("_", 1)[1])
    if args.workload.startswith("serving_"):
        return run_serving(args, args.workload.split("_", 1)[1])
    return run_ours(args)


def summarize(line):
    keep = ["metric", "value", "unit", "ms_per_step", "steps", "warmup", "dtype", "config", "error", "clocks",
            "step_ms", "latency_us", "offered_effective_tflops", "gpu_launches", "plain_f64_capacity"]
    out = {k: line[k] for k in keep if k in line}
    if line.get("roofline"):
        out["roofline"] = {k: line["roofline"][k] for k in ("bound", "achieved", "peak", "unit", "frac", "kernel")}
    if line.get("e2e"):
        out["e2e"] = line["e2e"]
    return out


def run_configs(args):
    import copy

    import torch
    out = []
    for label, wl, over in SUB_CONFIGS:
        sub = copy.copy(args)
        sub.workload = wl
        sub.steps = max(5, min(args.steps, 10))
        sub.warmup = 3
        sub.no_library = sub.no_cpu_baseline = sub.no_plain = True
        sub.cutoff = None
        for k, v in over.items():
            setattr(sub, k, v)
        try:
            res = summarize(dispatch(sub))
        except Exception as e:  # keep the headline line whatever happens here
            res = {"config": {"workload": wl}, "failed": repr(e)[:300]}
        res["label"] = label
        out.append(res)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + sorted(GEMM_WORKLOADS) + EXTRA_WORKLOADS,
                    default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-library", action="store_true", help="skip the torch.matmul library reference")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload only: skip the other workloads' short runs")
    ap.add_argument("--duration", type=float, default=10.0, help="serving: seconds of arrivals")
    ap.add_argument("--rate", type=float, default=2000.0,
                    help="serving: requests per second (at most the mode's measured-clean rate)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cutoff", type=int, default=None, help="override the workload's cutoff")
    ap.add_argument("--model-cutoff", action="store_true",
                    help="take the planner's cost-model cutoff instead of measuring candidates (ata_tune)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload.startswith("serving_"):
        mode = args.workload.split("_", 1)[1]
        if args.rate > SERVING_CLEAN_RATE.get(mode, 0.0):
            ap.error(f"--rate {args.rate:g} for {args.workload} is refused: measured-clean rates are "
                     f"{SERVING_CLEAN_RATE} requests per second")
    if args.impl == "reference":
        if args.workload not in WORKLOADS:
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the A^t A oracle on the "
                                                                  "A^t A workloads only"}))
            return 0
        return run_reference(args)
    line = dispatch(args)
    if line is None:
        return 0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.workload == DEFAULT_WORKLOAD and world == 1 and not args.no_configs:
        line["configs"] = run_configs(args)
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
