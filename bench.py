"""Benchmark: RLOBPCG solves/s on GB300 (one JSON line on rank 0).

Workload (default): m = 1e5, n = 500, k = 5, d = 3n, zeta = 8, FP64. Two seeded synthetic matrices
of the paper's structure, solved alternately: A = B C with an exact 5-dimensional nullspace, and a
planted spectrum with sigma_496..500 in [1e-12, 1e-9] below sigma_495 = 1e-4 (Haar U, V).
One step = one complete solve (sketch, QR, SVD of R, R^{-1}, start block, LOBPCG iterations with
the paper's stopping rule, outputs). A (400 MB) is larger than the 129 MB L2, so no flush is needed
between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own matrices on its own GPU (independent problems, no
collective on the data path: weak scaling); rank 0 prints the max-over-ranks time.
`--impl reference` times the CPU oracle (the plain numpy implementation of Algorithm 2 that the
tests check the GPU against) on a bounded row sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2602_16797_gb300 import replicas  # noqa: E402

METRIC = "solve time & solves/s at stated σ/angle error; fused AᴴAX GB/s; p50/p99 latency"
WORKLOAD = "nullspace+planted m=1e5 n=500 k=5 d=3n zeta=8 fp64"
M, N, K_TRIPLETS, D, ZETA = 100_000, 500, 5, 1500, 8
SAMPLE_M = 20_000          # row sample for the CPU oracle timings
FP64_UNITS_PER_SM_CLK = 2  # DFMA per clock per SM: 1.25 TFLOP/s nominal / (152 SMs * 2.07 GHz * 2 flop)


def make_inputs(m):
    from paper_2602_16797_gb300 import workloads as wl
    A0, _ = wl.exact_nullspace(m=m)
    A1, _, _ = wl.planted_bottom_cluster(m=m)
    return [A0, A1]


# ------------------------------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------- oracle timing

def oracle_solves_per_s(n_solves, warmup=0):
    """The oracle on the row-sampled workload; returns (full-size solves/s estimate, seconds, info)."""
    import oracle
    As = make_inputs(SAMPLE_M)
    for i in range(warmup):
        oracle.rlobpcg(As[i % 2], k=K_TRIPLETS, d=D, zeta=ZETA, seed=2002 + (i % 2))
    times = []
    for i in range(n_solves):
        t0 = time.perf_counter()
        oracle.rlobpcg(As[i % 2], k=K_TRIPLETS, d=D, zeta=ZETA, seed=2002 + (i % 2))
        times.append(time.perf_counter() - t0)
    per = sum(times) / len(times)
    # per-solve work of the method is proportional to m (sketch and every iteration stream A)
    return (SAMPLE_M / M) / per, times


def cpu_cores():
    return os.cpu_count() or 1


# --------------------------------------------------------------------------------------- our arm

def gram_traffic_per_element():
    """DRAM bytes per element of A per Gram pass from the committed ncu summary, if that summary
    was taken on the current gram.cu (else None)."""
    path = os.path.join(ROOT, "profiles", "gram_fused_ncu_summary.md")
    src = os.path.join(ROOT, "paper_2602_16797_gb300", "csrc", "gram.cu")
    try:
        txt = open(path).read()
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        tag, per = None, None
        for ln in txt.splitlines():
            if ln.startswith("gram.cu sha256[:16]: "):
                tag = ln.split(": ", 1)[1].strip()
            if ln.startswith("dram bytes per element of A: "):
                per = float(ln.split(": ", 1)[1].split()[0])
        return per if tag == h else None
    except (OSError, ValueError):
        return None


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2602_16797_gb300 import rlobpcg as rl

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    rl.load()
    As = make_inputs(M)
    Ad = [torch.from_numpy(A).to(dev) for A in As]
    stream = torch.cuda.current_stream(dev)
    o = rl.rlobpcg_default_opts()
    o.d = D
    o.zeta = ZETA
    plan = rl.rlobpcg_plan(M, N, K_TRIPLETS, rl.RLOBPCG_F64, o, stream.cuda_stream)
    sigma = torch.empty(K_TRIPLETS, dtype=torch.float64, device=dev)
    resid = torch.empty(K_TRIPLETS, dtype=torch.float64, device=dev)
    V = torch.empty((N, K_TRIPLETS), dtype=torch.float64, device=dev)

    def step(i, info):
        o.seed = 2002 + (i % 2)
        rl.rlobpcg_solve(plan, Ad[i % 2].data_ptr(), N, -1.0, sigma.data_ptr(), V.data_ptr(), None,
                         resid.data_ptr(), info)

    for i in range(args.warmup):
        step(i, rl.rlobpcg_info())
    torch.cuda.synchronize()
    replicas.barrier(world)
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    infos = []
    torch.cuda.synchronize()
    ev[0].record(stream)
    for i in range(args.steps):
        info = rl.rlobpcg_info()
        step(i, info)
        ev[i + 1].record(stream)
        infos.append(info)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_total = ev[0].elapsed_time(ev[-1])
    lat = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    replicas.barrier(world)
    ms_total = replicas.max_over_ranks(ms_total, world, device=dev)

    # e2e: host buffers through the same C-ABI call (H2D of A and D2H of the results inside)
    pinned = [torch.from_numpy(A).pin_memory() for A in As]
    sig_h = torch.empty(K_TRIPLETS, dtype=torch.float64).pin_memory()
    V_h = torch.empty((N, K_TRIPLETS), dtype=torch.float64).pin_memory()
    res_h = torch.empty(K_TRIPLETS, dtype=torch.float64).pin_memory()
    e2e_steps = max(2, min(args.steps, 4))
    info = rl.rlobpcg_info()
    o.seed = 2002
    rl.rlobpcg_solve(plan, pinned[0].data_ptr(), N, -1.0, sig_h.data_ptr(), V_h.data_ptr(), None, res_h.data_ptr(),
                     info)  # warm the plan's host-input buffer
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        o.seed = 2002 + (i % 2)
        rl.rlobpcg_solve(plan, pinned[i % 2].data_ptr(), N, -1.0, sig_h.data_ptr(), V_h.data_ptr(), None,
                         res_h.data_ptr(), info)
    e2e_s = time.perf_counter() - t0
    rl.rlobpcg_plan_destroy(plan)

    # roofline of the fused Gram pass (FP64 ALU bound): algorithmic flops per pass / event time
    gram_ms = sum(x.ms_gram for x in infos)
    passes = sum(x.gram_passes for x in infos)
    b = K_TRIPLETS
    flops_pass = 4.0 * M * N * b
    bytes_pass = 8.0 * M * N + 8.0 * M * b
    avg_s = gram_ms / max(passes, 1) * 1e-3
    achieved_tf = flops_pass / avg_s / 1e12 if passes else None
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    max_mhz = clk.get("sm_max_mhz") or 2070.0
    peak_tf = sm_count * FP64_UNITS_PER_SM_CLK * 2 * max_mhz * 1e6 / 1e12
    per_elem = gram_traffic_per_element()
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": (achieved_tf / peak_tf) if achieved_tf else None,
                "traffic": (per_elem * M * N) if per_elem is not None else None,
                "kernel": "gram_kernel (fused A W, A^H A W), FP64",
                "peak_source": f"derived: {sm_count} SMs x {FP64_UNITS_PER_SM_CLK} DFMA/clk x 2 flop x {max_mhz:.0f} MHz",
                "achieved_gbs": bytes_pass / avg_s / 1e9 if passes else None,
                "passes_timed": passes}

    out = None
    if rank == 0:
        ms_per = ms_total / args.steps
        value = replicas.job_rate(args.steps, world, ms_total * 1e-3)
        lat_sorted = sorted(lat)
        result = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded, paper-shaped; see DESIGN.md)",
            "config": {"workload": WORKLOAD, "m": M, "n": N, "k": K_TRIPLETS, "d": D, "zeta": ZETA,
                       "matrices": "exact nullspace A=BC and planted sigma_496..500 in [1e-12,1e-9], alternating",
                       "l2": "inputs (400 MB each) larger than L2; no flush", "parallelism": f"replicas x{world}"},
            "latency_ms": {"p50": float(np.percentile(lat_sorted, 50)), "p99": float(np.percentile(lat_sorted, 99))},
            "iters": [x.iters for x in infos], "stop_reasons": [x.stop_reason for x in infos],
            "jacobi_sweeps": [x.jacobi_sweeps for x in infos],
            "phase_ms": {"sketch": statistics.mean(x.ms_sketch for x in infos),
                         "factor": statistics.mean(x.ms_factor for x in infos),
                         "iterate": statistics.mean(x.ms_iterate for x in infos),
                         "gram_per_pass": avg_s * 1e3},
            "roofline": roofline, "clocks": clk,
            "gpu_launches": int(sum(x.kernel_launches for x in infos)),
            "e2e": {"value": e2e_steps / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": 8 * M * N,
                    "d2h_bytes_per_step": 8 * (K_TRIPLETS + N * K_TRIPLETS + K_TRIPLETS)},
        }
        if world == 1 and not args.no_cpu_baseline:
            v, times = oracle_solves_per_s(3)
            result["cpu_baseline"] = {"value": v, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                                      "sample": f"3 oracle solves of the same two matrix families at m={SAMPLE_M} "
                                                f"rows ({sum(times):.1f} s), scaled by {SAMPLE_M}/{M} (work is "
                                                f"linear in m); numpy/LAPACK with all host cores"}
        out = result
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    warm = args.warmup
    v, times = oracle_solves_per_s(args.steps, warmup=warm)
    total = sum(times)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": warm, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded, paper-shaped; see DESIGN.md)",
            "config": {"workload": WORKLOAD, "m": M, "n": N, "k": K_TRIPLETS, "d": D, "zeta": ZETA,
                       "parallelism": "cpu oracle, rank 0 only"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"each step one oracle solve at m={SAMPLE_M} rows, scaled by {SAMPLE_M}/{M}"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank, world, local_rank = replicas.world_from_env()
    if world > 1 and args.impl == "ours":
        import torch
        torch.cuda.set_device(local_rank)
    replicas.init(world, "nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local_rank)
    replicas.finish(world)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
