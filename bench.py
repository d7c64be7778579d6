"""Benchmark: RLOBPCG solves/s on GB300 (one JSON line on rank 0).

Workload (default): m = 1e5, n = 500, k = 5, d = 3n, zeta = 8, FP64. Two seeded synthetic matrices
of the paper's structure, solved alternately: A = B C with an exact 5-dimensional nullspace, and a
planted spectrum with sigma_496..500 in [1e-12, 1e-9] below sigma_495 = 1e-4 (Haar U, V).
One step = one complete solve (sketch, QR, SVD of R, R^{-1}, start block, LOBPCG iterations with
the paper's stopping rule, outputs). A (400 MB) is larger than the 129 MB L2, so no flush is needed
between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

--workload selects one of the other configurations of the study (small 4000 x 50, complex
2e5 x 300 with FP32 or FP64 sketch, 1e6 x 1000 FP64 or mixed); the default is the one above.

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
SAMPLE_FRAC = 0.2          # row sample of the CPU oracle timings (m -> 0.2 m)
FP64_UNITS_PER_SM_CLK = 2  # DFMA per clock per SM: 1.25 TFLOP/s nominal / (152 SMs * 2.07 GHz * 2 flop)


def _host_pair(m):
    from paper_2602_16797_gb300 import workloads as wl
    A0, _ = wl.exact_nullspace(m=m)
    A1, _, _ = wl.planted_bottom_cluster(m=m)
    return [A0, A1]


def _host_small(m):
    from paper_2602_16797_gb300 import workloads as wl
    return [wl.planted_small_gap_free(m=m)[0]]


def _host_complex(m):
    from paper_2602_16797_gb300 import workloads as wl
    return [wl.planted_complex(m=m)[0]]


def _device_large(m, device):
    from paper_2602_16797_gb300 import workloads as wl
    return [wl.planted_large_device(m=m, device=device)[0]]


# Named workloads. The default is the m = 1e5, n = 500, k = 5 configuration; the others are the
# remaining configurations of the same study (same JSON line, selected with --workload).
WORKLOADS = {
    "nullspace_1e5x500": dict(
        desc="nullspace+planted m=1e5 n=500 k=5 d=3n zeta=8 fp64", m=100_000, n=500, k=5, d=1500, zeta=8,
        cplx=False, prec=0, host=_host_pair, seeds=(2002, 2003),
        matrices="exact nullspace A=BC and planted sigma_496..500 in [1e-12,1e-9], alternating"),
    "small_4000x50": dict(
        desc="planted m=4000 n=50 k=1 d=4n zeta=8 tau=1e-12 fp64", m=4000, n=50, k=1, d=200, zeta=8, cplx=False,
        prec=0, host=_host_small, seeds=(1001,), tau=1e-12, stagnation=0,
        matrices="planted sigma_1..49 logspace(0,-6), sigma_50=1e-10"),
    "complex_2e5x300_f32sketch": dict(
        desc="complex planted m=2e5 n=300 k=3 d=4n zeta=8 fp32 sketch", m=200_000, n=300, k=3, d=1200, zeta=8,
        cplx=True, prec=1, host=_host_complex, seeds=(1003,),
        matrices="complex planted sigma logspace(0,-8), three smallest 1e-12, 3e-13, 1e-13"),
    "complex_2e5x300": dict(
        desc="complex planted m=2e5 n=300 k=3 d=4n zeta=8 fp64 sketch", m=200_000, n=300, k=3, d=1200, zeta=8,
        cplx=True, prec=0, host=_host_complex, seeds=(1003,),
        matrices="complex planted sigma logspace(0,-8), three smallest 1e-12, 3e-13, 1e-13"),
    "large_1e6x1000_mixed": dict(
        desc="planted m=1e6 n=1000 k=10 d=4n zeta=8 fp32 sketch/R, fp64 Gram", m=1_000_000, n=1000, k=10, d=4000,
        zeta=8, cplx=False, prec=1, device=_device_large, seeds=(1004,),
        matrices="planted sigma_1..990 logspace(0,-4), sigma_991..1000 logspace(-9,-10)"),
    "large_1e6x1000": dict(
        desc="planted m=1e6 n=1000 k=10 d=4n zeta=8 fp64", m=1_000_000, n=1000, k=10, d=4000, zeta=8,
        cplx=False, prec=0, device=_device_large, seeds=(1004,),
        matrices="planted sigma_1..990 logspace(0,-4), sigma_991..1000 logspace(-9,-10)"),
}
DEFAULT_WORKLOAD = "nullspace_1e5x500"


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

def oracle_solves_per_s(w, n_solves, warmup=0):
    """The oracle on a row sample (m -> SAMPLE_FRAC m) of the workload; returns (full-size solves/s
    estimate, per-solve seconds). Per-solve work is linear in m (the sketch and every iteration
    stream A once)."""
    import oracle
    ms = int(w["m"] * SAMPLE_FRAC)
    if "host" in w:
        As = w["host"](ms)
    else:
        from paper_2602_16797_gb300 import workloads as wl
        sig = np.concatenate([np.logspace(0, -4, w["n"] - w["k"]), np.logspace(-9, -10, w["k"])])
        As = [wl.planted(np.random.default_rng(w["seeds"][0]), ms, sig)[0]]
    kw = dict(k=w["k"], d=w["d"], zeta=w["zeta"], sketch_precision="f32" if w["prec"] else "f64")
    if "tau" in w:
        kw["tau"] = w["tau"]
    if w.get("stagnation", 1) == 0:
        kw["use_stagnation"] = False
    for i in range(warmup):
        oracle.rlobpcg(As[i % len(As)], seed=w["seeds"][i % len(w["seeds"])], **kw)
    times = []
    for i in range(n_solves):
        t0 = time.perf_counter()
        oracle.rlobpcg(As[i % len(As)], seed=w["seeds"][i % len(w["seeds"])], **kw)
        times.append(time.perf_counter() - t0)
    per = sum(times) / len(times)
    return (ms / w["m"]) / per, times


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def cpu_cores():
    return os.cpu_count() or 1


def oracle_rate_one_thread(workload, n_solves=1, timeout=300):
    """The same oracle sample with every BLAS/OpenMP pool at one thread, in a fresh interpreter
    (the pools of this process are already sized); None if it cannot be measured."""
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
                "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[var] = "1"
    code = ("import json, bench; v, t = bench.oracle_solves_per_s(bench.WORKLOADS[%r], %d); "
            "print(json.dumps([v, sum(t)]))" % (workload, n_solves))
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=timeout)
        v, secs = json.loads(r.stdout.strip().splitlines()[-1])
        return float(v), float(secs)
    except (subprocess.SubprocessError, ValueError, IndexError, OSError):
        return None


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


def split_traffic_per_launch(m, n, k):
    """DRAM bytes per launch of the two split-Gram kernels (A W and A^T (A W)) from the committed ncu
    summary, scaled to (m, n) by the digit bytes, if that summary was taken on the current
    gram_tc.cu (else None)."""
    path = os.path.join(ROOT, "profiles", "gram_split_ncu_summary.md")
    src = os.path.join(ROOT, "paper_2602_16797_gb300", "csrc", "gram_tc.cu")
    try:
        txt = open(path).read()
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        tag, per = None, {}
        for ln in txt.splitlines():
            if ln.startswith("gram_tc.cu sha256[:16]: "):
                tag = ln.split(": ", 1)[1].strip()
            for key in ("ab", "atb"):
                pre = f"dram bytes per digit byte ({key}): "
                if ln.startswith(pre):
                    per[key] = float(ln.split(": ", 1)[1].split()[0])
        if tag != h or len(per) != 2:
            return None
        alg = split_algorithmic_bytes(m, n, k)
        return {key: per[key] * alg[key + "_digits"] for key in ("ab", "atb")}
    except (OSError, ValueError):
        return None


def split_algorithmic_bytes(m, n, b):
    """Bytes each split-Gram kernel must move per launch (layouts of gram_tc.cu): the digits of A
    (8 one-byte digits per element of the padded matrix, as many bytes as the FP64 value), plus
    A W (FP64) and the bf16 digits of A W (8 x 8 or 8 x 16 per row) written by the first, read by
    the second once per 128-column tile."""
    cd = lambda a, q: -(-a // q)  # noqa: E731
    R1, NKB, CT = cd(m, 128), cd(n, 16), cd(n, 128)
    N = 8 * (8 if b <= 8 else 16)
    tile = 128 * 16 * 8
    ab_digits = R1 * NKB * tile
    atb_digits = CT * R1 * 8 * tile
    y_digits = R1 * 128 * N * 2
    return {"ab_digits": ab_digits, "atb_digits": atb_digits,
            "ab": ab_digits + 8 * m * b + y_digits, "atb": atb_digits + CT * y_digits}


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2602_16797_gb300 import rlobpcg as rl

    w = WORKLOADS[args.workload]
    M, N, K, D = w["m"], w["n"], w["k"], w["d"]
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    rl.load()
    if "host" in w:
        hostA = w["host"](M)
        Ad = [torch.from_numpy(A).to(dev) for A in hostA]
    else:
        Ad = w["device"](M, dev)
        hostA = None
    dtype = rl.RLOBPCG_C128 if w["cplx"] else rl.RLOBPCG_F64
    tdt = torch.complex128 if w["cplx"] else torch.float64
    esz = 16 if w["cplx"] else 8
    stream = torch.cuda.current_stream(dev)
    o = rl.rlobpcg_default_opts()
    o.d = D
    o.zeta = w["zeta"]
    o.sketch_prec = w["prec"]
    o.gram_split = 1 if args.gram == "split" else 0
    split = args.gram == "split" and not w["cplx"] and K <= 16
    if "stagnation" in w:
        o.use_stagnation = w["stagnation"]
    if "tau" in w:
        o.tau = w["tau"]
    plan = rl.rlobpcg_plan(M, N, K, dtype, o, stream.cuda_stream)
    sigma = torch.empty(K, dtype=torch.float64, device=dev)
    resid = torch.empty(K, dtype=torch.float64, device=dev)
    V = torch.empty((N, K), dtype=tdt, device=dev)
    seeds = w["seeds"]

    def step(i, info, A_ptr=None, out=None):
        o.seed = seeds[i % len(seeds)]
        a = A_ptr if A_ptr is not None else Ad[i % len(Ad)].data_ptr()
        sg, vv, rs = out if out is not None else (sigma.data_ptr(), V.data_ptr(), resid.data_ptr())
        rl.rlobpcg_solve(plan, a, N, -1.0, sg, vv, None, rs, info)

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
    pinned = [torch.from_numpy(A).pin_memory() for A in hostA] if hostA is not None else \
        [A.cpu().pin_memory() for A in Ad]
    sig_h = torch.empty(K, dtype=torch.float64).pin_memory()
    V_h = torch.empty((N, K), dtype=tdt).pin_memory()
    res_h = torch.empty(K, dtype=torch.float64).pin_memory()
    hout = (sig_h.data_ptr(), V_h.data_ptr(), res_h.data_ptr())
    e2e_steps = max(2, min(args.steps, 4))
    info = rl.rlobpcg_info()
    step(0, info, pinned[0].data_ptr(), hout)  # warm the plan's host-input buffer
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        step(i, info, pinned[i % len(pinned)].data_ptr(), hout)
    e2e_s = time.perf_counter() - t0
    rl.rlobpcg_plan_destroy(plan)

    # roofline of the fused Gram pass (FP64 ALU bound): algorithmic flops per pass / event time
    gram_ms = sum(x.ms_gram for x in infos)
    passes = sum(x.gram_passes for x in infos)
    fl_el = 16.0 if w["cplx"] else 4.0
    flops_pass = fl_el * M * N * K
    bytes_pass = esz * (M * N + M * K)
    avg_s = gram_ms / max(passes, 1) * 1e-3
    achieved_tf = flops_pass / avg_s / 1e12 if passes else None
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    max_mhz = clk.get("sm_max_mhz") or 2070.0
    peak_tf = sm_count * FP64_UNITS_PER_SM_CLK * 2 * max_mhz * 1e6 / 1e12
    if split:
        # split-bf16 Gram: two tensor-core kernels per pass that stream the byte digits of A; the
        # roofline is that of the slower one (bytes it must move per launch / its event-timed
        # duration) against the measured copy bandwidth
        alg = split_algorithmic_bytes(M, N, K)
        t_ab = sum(x.ms_gram_ab for x in infos) / max(passes, 1) * 1e-3
        t_atb = sum(x.ms_gram_atb for x in infos) / max(passes, 1) * 1e-3
        key, t_k = ("atb", t_atb) if t_atb >= t_ab else ("ab", t_ab)
        peaks = measured_peaks()
        peak_gbs = peaks.get("hbm_gbs") or 6800.0
        achieved_gbs = alg[key] / t_k / 1e9 if passes else None
        tr = split_traffic_per_launch(M, N, K)
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": peak_gbs, "unit": "GB/s",
                    "frac": (achieved_gbs / peak_gbs) if achieved_gbs else None,
                    "traffic": tr[key] if tr else None,
                    "kernel": ("split_pass_kernel<8,1> (A^T (A W), byte digits expanded to bf16 in TMEM, tcgen05)"
                               if key == "atb" else
                               "split_pass_kernel<8,0> (A W, byte digits expanded to bf16 in TMEM, tcgen05)"),
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks.get("hbm_gbs") else
                                   "fallback 6.8 TB/s",
                    "bytes_per_launch": alg[key], "ms_per_launch": t_k * 1e3,
                    "other_kernel_ms": (t_ab if key == "atb" else t_atb) * 1e3,
                    "gram_pass_fp64_equiv_tflops": achieved_tf, "passes_timed": passes}
    else:
        per_elem = gram_traffic_per_element() if args.workload == DEFAULT_WORKLOAD else None
        roofline = {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                    "frac": (achieved_tf / peak_tf) if achieved_tf else None,
                    "traffic": (per_elem * M * N) if per_elem is not None else None,
                    "kernel": "gram_kernel (fused A W, A^H A W), " + ("complex128" if w["cplx"] else "FP64"),
                    "peak_source": f"derived: {sm_count} SMs x {FP64_UNITS_PER_SM_CLK} DFMA/clk x 2 flop x {max_mhz:.0f} MHz",
                    "achieved_gbs": bytes_pass / avg_s / 1e9 if passes else None,
                    "passes_timed": passes}

    out = None
    if rank == 0:
        ms_per = ms_total / args.steps
        value = replicas.job_rate(args.steps, world, ms_total * 1e-3)
        result = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128" if w["cplx"] else "f64",
            "data": "synthetic (seeded; the paper's matrix families)",
            "config": {"workload": w["desc"], "m": M, "n": N, "k": K, "d": D, "zeta": w["zeta"],
                       "sketch": "fp32" if w["prec"] else "fp64", "matrices": w["matrices"],
                       "gram": "split-bf16 tensor cores" if split else ("fp64 CUDA cores" if not w["cplx"]
                                                                         else "complex128 CUDA cores"),
                       "l2": "input larger than L2; no flush" if M * N * esz > 129e6 else
                             "input smaller than L2 (each step is a full solve)",
                       "parallelism": f"replicas x{world}"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "iters": [x.iters for x in infos], "stop_reasons": [x.stop_reason for x in infos],
            "rr_sweeps_per_svd": round(sum(x.rr_sweeps for x in infos) / max(1, sum(x.rr_calls for x in infos)), 2),
            "phase_ms": {"sketch": statistics.mean(x.ms_sketch for x in infos),
                         "factor": statistics.mean(x.ms_factor for x in infos),
                         "iterate": statistics.mean(x.ms_iterate for x in infos),
                         "gram_per_pass": avg_s * 1e3,
                         "per_iteration": statistics.mean(x.ms_iterate / max(x.iters, 1) for x in infos),
                         "split_a": statistics.mean(x.ms_split_a for x in infos)},
            "sigma": [float(x) for x in sigma.cpu().numpy()],
            "roofline": roofline, "clocks": clk,
            "gpu_launches": int(sum(x.kernel_launches for x in infos)),
            "e2e": {"value": e2e_steps / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": esz * M * N,
                    "d2h_bytes_per_step": 8 * K + esz * N * K + 8 * K},
        }
        if world == 1 and not args.no_cpu_baseline:
            v, times = oracle_solves_per_s(w, 3)
            result["cpu_baseline"] = {"value": v, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                                      "sample": f"3 oracle solves of the same matrix families at m={int(M * SAMPLE_FRAC)} "
                                                f"rows ({sum(times):.1f} s), scaled by {SAMPLE_FRAC} (work is linear "
                                                f"in m); numpy/LAPACK with all host cores"}
            one = oracle_rate_one_thread(args.workload)
            if one is not None:
                result["cpu_baseline"]["value_1_thread"] = one[0]
                result["cpu_baseline"]["sample"] += f"; value_1_thread: one such solve with one thread ({one[1]:.1f} s)"
        out = result
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    w = WORKLOADS[args.workload]
    v, times = oracle_solves_per_s(w, args.steps, warmup=args.warmup)
    total = sum(times)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128" if w["cplx"] else "f64", "data": "synthetic (seeded; the paper's matrix families)",
            "config": {"workload": w["desc"], "m": w["m"], "n": w["n"], "k": w["k"], "d": w["d"], "zeta": w["zeta"],
                       "parallelism": "cpu oracle, rank 0 only"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"each step one oracle solve at m={int(w['m'] * SAMPLE_FRAC)} rows, "
                                       f"scaled by {SAMPLE_FRAC}"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_serve(args, rank, world, local_rank):
    """Serving stream: half Loewner, half planted requests (m log-uniform in [2e3, 5e5], n uniform
    in [20, 400], k in {1, 2, 4}), HBM admission budget 150 GB. Measures the saturated rate with
    `--slots` concurrent solves, the same stream one solve at a time, and Poisson arrivals at
    0.5 / 0.9 / 1.2 x the saturated rate (p50 / p99 latency from submit to result)."""
    import torch

    from paper_2602_16797_gb300 import rlobpcg as rl
    from paper_2602_16797_gb300 import workloads as wl
    if rank != 0:
        return None
    torch.cuda.set_device(local_rank)
    rl.load()
    reqs = []
    for r in range(args.requests):
        A, k, kind = wl.serve_request(r)
        reqs.append((np.ascontiguousarray(A), k, wl.SERVE_SEED_BASE + r))
    budget = 150 * (1 << 30)

    def opts(seed):
        o = rl.rlobpcg_default_opts()
        o.seed = seed
        return o

    def stream(slots, arrivals=None):
        srv = rl.rlobpcg_server_create(budget, slots, local_rank)
        t0 = time.perf_counter()
        tickets = []
        for i, (A, k, seed) in enumerate(reqs):
            if arrivals is not None:
                dt = t0 + arrivals[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            tickets.append(rl.rlobpcg_server_submit(srv, A.ctypes.data, A.shape[0], A.shape[1], A.shape[1], k,
                                                    rl.RLOBPCG_F64, opts(seed)))
        iters = []
        for (A, k, seed), t in zip(reqs, tickets):
            info = rl.rlobpcg_info()
            rl.rlobpcg_server_wait(srv, t, None, None, None, info)
            iters.append(info.iters)
        makespan = time.perf_counter() - t0
        st = rl.rlobpcg_server_stats(srv)
        rl.rlobpcg_server_destroy(srv)
        st["makespan_s"] = makespan
        st["rate"] = len(reqs) / makespan
        st["mean_iters"] = float(np.mean(iters))
        return st

    warm = reqs[:4]
    for A, k, seed in warm:
        rl.solve(torch.from_numpy(A).cuda(), k, opts=opts(seed))
    sat = stream(args.slots)
    seq = stream(1)
    lat = {}
    rng = np.random.default_rng(4242)
    for f in (0.5, 0.9, 1.2):
        lam = f * sat["rate"]
        arr = np.cumsum(rng.exponential(1.0 / lam, len(reqs)))
        st = stream(args.slots, arr)
        lat[f"{f}x"] = {"offered_per_s": lam, "solves_per_s": st["rate"], "p50_ms": st["p50_ms"],
                        "p99_ms": st["p99_ms"], "peak_running": st["peak_running"], "peak_gb": st["peak_bytes"] / 1e9}
    bytes_in = float(np.mean([A.nbytes for A, _, _ in reqs]))
    return {"metric": METRIC, "value": sat["rate"], "unit": "solves/s", "n_gpus": 1, "steps": len(reqs),
            "warmup": len(warm), "ms_per_step": 1e3 / sat["rate"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded; the paper's matrix families)",
            "config": {"workload": f"serving stream of {len(reqs)} requests (half Loewner, half planted; m log-uniform "
                                   f"[2e3,5e5], n U[20,400], k in {{1,2,4}}), HBM budget 150 GB, {args.slots} slots",
                       "parallelism": "continuous batching on one GPU"},
            "saturated": {"solves_per_s": sat["rate"], "p50_ms": sat["p50_ms"], "p99_ms": sat["p99_ms"],
                          "peak_running": sat["peak_running"], "mean_iters": sat["mean_iters"]},
            "one_at_a_time": {"solves_per_s": seq["rate"], "p50_ms": seq["p50_ms"], "p99_ms": seq["p99_ms"]},
            "poisson": lat,
            "e2e": {"value": sat["rate"], "unit": "solves/s", "h2d_bytes_per_step": bytes_in,
                    "d2h_bytes_per_step": None}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["serve_stream"], default=DEFAULT_WORKLOAD)
    ap.add_argument("--gram", choices=["split", "fp64"], default="split",
                    help="Gram products: split-bf16 on the tensor cores (default) or FP64 CUDA cores")
    ap.add_argument("--requests", type=int, default=48, help="serve_stream: number of requests")
    ap.add_argument("--slots", type=int, default=8, help="serve_stream: concurrent solves")
    args = ap.parse_args()
    rank, world, local_rank = replicas.world_from_env()
    if world > 1 and args.impl == "ours":
        import torch
        torch.cuda.set_device(local_rank)
    replicas.init(world, "nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload == "serve_stream":
        out = run_serve(args, rank, world, local_rank)
    else:
        out = run_ours(args, rank, world, local_rank)
    replicas.finish(world)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
