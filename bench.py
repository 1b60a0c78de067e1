#!/usr/bin/env python
"""Benchmark of C = A^t A on one GB300 (or N replicas under torchrun).

Default workload: plain FP64 ATA at the paper's scale, A 10000 x 10000 with
i.i.d. N(0, 1) entries from seed 1, cutoff chosen by the planner's autotuner,
packed upper-triangle FP64 output.  A step is one ata_execute (one replay of
the plan's CUDA graph: operand splits, the persistent leaf launch, Strassen
combines) over the resident input.  The metric is effective TFLOP/s =
2 m n^2 / t (m n^2 classical FMAs), at the componentwise error reported in
the line.

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
}
MODE_CODES = {"f64": 0, "bf16x3": 1, "tf32": 2, "ozaki": 3}
PAIRS = {"f64": 1, "bf16x3": 6, "tf32": 1, "ozaki": 21}
TOLERANCE = {"f64": ("componentwise", 1e-11), "ozaki": ("componentwise", 1e-11),
             "bf16x3": ("normwise", 1e-6), "tf32": ("normwise", 1e-3)}
DEFAULT_WORKLOAD = "ata_f64_10000x10000"

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

# DRAM traffic of the leaf kernel from one ncu capture, per launch, valid only
# for the kernel source it was taken on (sha256 of kernels_f64.cu).
LEAF_TRAFFIC = {}


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
    if world == 1:
        return value
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_oracle_sample(A, budget_s=15.0):
    """Times the oracle on leading rows of the packed triangle for about
    budget_s seconds and extrapolates to the whole product."""
    import oracle
    m, n = A.shape
    total = m * n * (n + 1) / 2
    # calibrate on a few rows
    rows = max(1, min(n, 16))
    t0 = time.perf_counter()
    oracle.ata_rows(A, 0, rows)
    dt = time.perf_counter() - t0
    done = m * sum(n - i for i in range(rows))
    rate = done / max(dt, 1e-6)
    # grow to the budget
    want = rate * budget_s
    r1 = rows
    acc = 0
    while r1 < n and acc < want:
        acc += m * (n - r1)
        r1 += 1
    t0 = time.perf_counter()
    oracle.ata_rows(A, rows, r1)
    dt = time.perf_counter() - t0
    done = m * sum(n - i for i in range(rows, r1))
    t_full = dt * total / max(done, 1)
    return {"t_full_s": t_full, "rows": (rows, r1), "sample_s": dt, "cores": oracle.num_threads(),
            "frac": done / total}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    name = args.workload
    m, n, mode, gen, seed, cutoff = WORKLOADS[name]
    A = make_input(name)
    eff = effective_flops(m, n)
    # each step: a bounded sample (~budget seconds) of the oracle
    budget = max(2.0, min(15.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_sample(A, budget_s=budget / 4)
    ts = []
    samples = []
    for _ in range(args.steps):
        r = cpu_oracle_sample(A, budget_s=budget)
        ts.append(r["t_full_s"])
        samples.append(r)
    t = statistics.median(ts)
    value = eff / t / 1e12
    last = samples[-1]
    line = {
        "impl": "reference", "metric": "effective TFLOP/s (m*n^2 FMAs) of C = A^t A", "value": value,
        "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "m": m, "n": n, "generator": f"{gen}(seed={seed})"},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": last["cores"], "kind": "oracle",
                         "sample": f"packed rows {last['rows'][0]}..{last['rows'][1]} "
                                   f"({100 * last['frac']:.2f}% of the multiplications) per step, "
                                   f"extrapolated to the whole product"},
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
    leaf_ms, split_ms, comb_ms, prep_ms = [], [], [], []
    e0.record(stream)
    for _ in range(args.steps):
        plan(A, C)
        stream.synchronize()
        st = plan.stage_times()
        leaf_ms.append(st["leaf_ms"])
        split_ms.append(st["split_ms"])
        prep_ms.append(st["prep_ms"])
        comb_ms.append(st["combine_ms"])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(torch, ms, world)

    # accuracy at the stated tolerance: sampled entries against the oracle
    err_kind, tol = TOLERANCE[mode]
    cnt = 2000
    err = sampled_error(oracle, A_np, C, n, err_kind, dev, torch, count=cnt)
    dev_status = plan.device_status()

    # end to end through the C ABI from pinned host memory
    A_host = torch.from_numpy(A_np).pin_memory()
    C_host = torch.empty(n * (n + 1) // 2, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    ata.ata_execute_host(plan, A_host.numpy(), C_host.numpy(), stream)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ata.ata_execute_host(plan, A_host.numpy(), C_host.numpy(), stream)
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
        "config": {"workload": name, "m": m, "n": n, "leaf": mode, "generator": f"{gen}(seed={seed})",
                   "cutoff": info["cutoff"],
                   "strassen_levels_max": info["max_strassen_levels"], "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (A is %d MB)" % (A_np.nbytes >> 20)},
        "error": {err_kind + "_sampled": err, "tolerance": tol, "samples": cnt, "device_status": dev_status},
        "stages_ms": {"split": statistics.mean(split_ms), "prep": statistics.mean(prep_ms),
                      "leaf": statistics.mean(leaf_ms), "combine": statistics.mean(comb_ms)},
        "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": tr, "peak_source": peak_src,
                     "kernel": kern, "flops_per_launch": leaf_flops},
        "e2e": {"value": world * eff / t_e2e / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": int(A_np.nbytes),
                "d2h_bytes_per_step": int(C.numel() * 8)},
        "gpu_launches": int(args.steps * info["n_launches"]),
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = cpu_oracle_sample(A_np, budget_s=args.cpu_budget)
        line["cpu_baseline"] = {
            "value": eff / r["t_full_s"] / 1e12, "unit": "TFLOP/s", "cores": r["cores"], "kind": "oracle",
            "sample": f"packed rows {r['rows'][0]}..{r['rows'][1]} ({100 * r['frac']:.2f}% of the "
                      f"multiplications, {r['sample_s']:.1f} s), extrapolated to the whole product"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cutoff", type=int, default=None, help="override the workload's cutoff")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
