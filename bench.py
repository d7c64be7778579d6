"""Benchmark: RLOBPCG solves/s on GB300 (one JSON line on rank 0).

Workload (default): the large planted configuration m = 1e6, n = 1000, k = 10, d = 4n, zeta = 8,
FP64 A of 8 GB (sigma_1..990 logspace(0,-4), sigma_991..1000 logspace(-9,-10), Haar U and V; built
on the GPU from a seeded Philox Gaussian). One step = one complete solve (sketch, QR, start block,
LOBPCG iterations with the paper's stopping rule, outputs). A (8 GB) is far larger than the
129 MB L2, so no flush is needed between steps. The line also carries the mixed-precision form
(`mixed`: FP32 sketch and R refined once in FP64) timed on the same matrix.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
                  [--fixed-iters I]

--workload selects one of the other configurations of the study (4000 x 50, 1e5 x 500 exact
nullspace + planted cluster, complex 2e5 x 300, the clustered 1e6 x 2000 block-size study, the
serving stream); --fixed-iters runs exactly I LOBPCG iterations per solve (no stop test), which
makes the per-iteration time independent of where the stopping rule fires.

Under torchrun each rank solves its own matrices on its own GPU (independent problems, no
collective on the data path: weak scaling); rank 0 prints the max-over-ranks time.
`--impl reference` times the CPU oracle (the plain numpy implementation of Algorithm 2 that the
tests check the GPU against) per phase on a bounded row sample of the same matrix family and
scales it to the full size.
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
FP64_UNITS_PER_SM_CLK = 2  # DFMA per clock per SM: 1.25 TFLOP/s nominal / (152 SMs * 2.07 GHz * 2 flop)
DIGIT_PAIRS = 43           # digit pairs per product of the split-bf16 Gram pass (levels p + q <= 8 of 8 x 8)


def _host_pair(m):
    from paper_2602_16797_gb300 import workloads as wl
    A0, _ = wl.exact_nullspace(m=m)
    A1, s1, _ = wl.planted_bottom_cluster(m=m)
    return [A0, A1], [np.zeros(5), np.sort(s1)[:5]]


def _host_small(m):
    from paper_2602_16797_gb300 import workloads as wl
    A, s, _ = wl.planted_small_gap_free(m=m)
    return [A], [np.sort(s)[:1]]


def _host_complex(m):
    from paper_2602_16797_gb300 import workloads as wl
    A, s, _ = wl.planted_complex(m=m)
    return [A], [np.sort(s)[:3]]


def _large_sigma(n=1000, k=10):
    return np.concatenate([np.logspace(0, -4, n - k), np.logspace(-9, -10, k)])


def _device_large(m, device):
    from paper_2602_16797_gb300 import workloads as wl
    A, s, _ = wl.planted_large_device(m=m, device=device)
    return [A], [np.sort(s)[:10]]


def _host_large_sample(m):
    """The same spectrum as the 1e6 x 1000 matrix on a row sample (host, for the CPU oracle)."""
    from paper_2602_16797_gb300 import workloads as wl
    A, s, _ = wl.planted_large(m=m)
    return [A], [np.sort(s)[:10]]


def _host_complex_sample(m):
    return _host_complex(m)


# Named workloads: the configurations of the study (same JSON line, selected with --workload).
# `sample_m` is the row count of the CPU oracle's sample; `host_sample` builds it.
WORKLOADS = {
    "large_1e6x1000": dict(
        desc="planted m=1e6 n=1000 k=10 d=4n zeta=8 fp64", m=1_000_000, n=1000, k=10, d=4000,
        zeta=8, cplx=False, prec=0, device=_device_large, seeds=(1004,), mixed_prec=2,
        host_sample=_host_large_sample, sample_m=100_000, ref_sample_m=20_000,
        matrices="planted sigma_1..990 logspace(0,-4), sigma_991..1000 logspace(-9,-10), Haar U, V"),
    "profile_2e5x1000": dict(
        desc="planted m=2e5 n=1000 k=10 d=4n zeta=8 fp64 (the 1e6 x 1000 recipe on 2e5 rows, for profiling)",
        m=200_000, n=1000, k=10, d=4000, zeta=8, cplx=False, prec=0, device=_device_large, seeds=(1004,),
        host_sample=_host_large_sample, sample_m=20_000, ref_sample_m=20_000,
        matrices="planted sigma_1..990 logspace(0,-4), sigma_991..1000 logspace(-9,-10), Haar U, V"),
    "nullspace_1e5x500": dict(
        desc="nullspace+planted m=1e5 n=500 k=5 d=3n zeta=8 fp64", m=100_000, n=500, k=5, d=1500, zeta=8,
        cplx=False, prec=0, host=_host_pair, seeds=(2002, 2003), sample_m=20_000,
        matrices="exact nullspace A=BC and planted sigma_496..500 in [1e-12,1e-9], alternating"),
    "small_4000x50": dict(
        desc="planted m=4000 n=50 k=1 d=4n zeta=8 tau=1e-12 fp64", m=4000, n=50, k=1, d=200, zeta=8, cplx=False,
        prec=0, host=_host_small, seeds=(1001,), tau=1e-12, stagnation=0, sample_m=4000,
        matrices="planted sigma_1..49 logspace(0,-6), sigma_50=1e-10"),
    "complex_2e5x300": dict(
        desc="complex planted m=2e5 n=300 k=3 d=4n zeta=8 fp64 sketch", m=200_000, n=300, k=3, d=1200, zeta=8,
        cplx=True, prec=0, host=_host_complex, seeds=(1003,), mixed_prec=2, sample_m=40_000,
        host_sample=_host_complex_sample,
        matrices="complex planted sigma logspace(0,-8), three smallest 1e-12, 3e-13, 1e-13"),
    "complex_2e5x300_f32sketch": dict(
        desc="complex planted m=2e5 n=300 k=3 d=4n zeta=8 fp32 sketch", m=200_000, n=300, k=3, d=1200, zeta=8,
        cplx=True, prec=1, host=_host_complex, seeds=(1003,), sample_m=40_000, host_sample=_host_complex_sample,
        matrices="complex planted sigma logspace(0,-8), three smallest 1e-12, 3e-13, 1e-13"),
}
DEFAULT_WORKLOAD = "large_1e6x1000"


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

def _oracle_kwargs(w):
    kw = dict(k=w["k"], d=w["d"], zeta=w["zeta"], sketch_precision="f32" if w["prec"] == 1 else "f64")
    if "tau" in w:
        kw["tau"] = w["tau"]
    if w.get("stagnation", 1) == 0:
        kw["use_stagnation"] = False
    return kw


_SAMPLE_CACHE = {}


def _sample_matrix(w, ms):
    """The row sample (ms rows of the workload's matrix family), built once per process."""
    key = (w["desc"], ms)
    if key not in _SAMPLE_CACHE:
        build = w.get("host_sample") or w["host"]
        As, _ = build(ms)
        _SAMPLE_CACHE[key] = As[0]
    return _SAMPLE_CACHE[key]


def oracle_sample_phases(w, run_to_stop=True, sample_m=None):
    """Time the CPU oracle, as it stands, on a row sample of the workload (m -> sample_m rows of the
    same matrix family and spectrum). Returns the seconds of its one-time part (sketch, SVD of the
    sketch, start block) split into the part that streams A (scales with m) and the SVD of the
    d x n sketch (does not), the seconds per LOBPCG iteration (every iteration streams A: scales
    with m), and the iteration count at which the oracle's own stopping rule fires on the sample."""
    import oracle
    ms = min(sample_m or w["sample_m"], w["m"])
    A = _sample_matrix(w, ms)
    seed = w["seeds"][0]
    kw = _oracle_kwargs(w)
    t0 = time.perf_counter()
    SA = oracle.sketch(A.astype(np.complex128 if w["cplx"] else np.float64), w["d"], w["zeta"], seed,
                       kw["sketch_precision"])
    t1 = time.perf_counter()
    oracle.sketch_svd(SA)
    t_svd = time.perf_counter() - t1
    t0 = time.perf_counter()
    oracle.rlobpcg(A, seed=seed, fixed_iters=1, **kw)
    t_fix1 = time.perf_counter() - t0
    t_fix3 = None
    stop_iters = None
    if run_to_stop:
        t0 = time.perf_counter()
        r = oracle.rlobpcg(A, seed=seed, **kw)
        t_stop = time.perf_counter() - t0
        stop_iters = int(r["iters"])
        t_iter = (t_stop - t_fix1) / max(stop_iters - 1, 1)
    else:
        t0 = time.perf_counter()
        oracle.rlobpcg(A, seed=seed, fixed_iters=3, **kw)
        t_fix3 = time.perf_counter() - t0
        t_iter = (t_fix3 - t_fix1) / 2.0
    t_once = max(t_fix1 - t_iter, t_svd)
    return {"sample_m": ms, "t_svd": t_svd, "t_once_stream": max(t_once - t_svd, 0.0), "t_iter": max(t_iter, 0.0),
            "stop_iters": stop_iters, "cpu_seconds": None}


def oracle_full_solve_seconds(w, ph, iters):
    """Full-size oracle solve time estimated from the sample's phases: the parts that stream A
    scale with m / sample_m, the SVD of the d x n sketch does not."""
    f = w["m"] / ph["sample_m"]
    return ph["t_once_stream"] * f + ph["t_svd"] + iters * ph["t_iter"] * f


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def cpu_cores():
    return os.cpu_count() or 1


def oracle_rate_one_thread(workload, iters, timeout=300):
    """The same oracle sample with every BLAS/OpenMP pool at one thread, in a fresh interpreter
    (the pools of this process are already sized): estimated full-size solves/s at `iters`
    iterations and the seconds the sample took; None if it cannot be measured in time."""
    env = dict(os.environ)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
                "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[var] = "1"
    code = ("import json, time, bench; w = bench.WORKLOADS[%r]; t0 = time.perf_counter(); "
            "ph = bench.oracle_sample_phases(w, run_to_stop=False); "
            "print(json.dumps([1.0 / bench.oracle_full_solve_seconds(w, ph, %d), time.perf_counter() - t0]))"
            % (workload, iters))
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=timeout)
        v, secs = json.loads(r.stdout.strip().splitlines()[-1])
        return float(v), float(secs)
    except (subprocess.SubprocessError, ValueError, IndexError, OSError, KeyError):
        return None


# --------------------------------------------------------------------------------- roofline helpers

def sigma_err(sig, truth, sigma11):
    """max_j |sigma_j - sigma_true_j| / max(sigma_true_j, Sigma~(1,1) 2^-52): relative to the planted
    value, or, where that is below what a backward-stable solve resolves (an exact nullspace has
    sigma_true = 0), in units of Sigma~(1,1) 2^-52."""
    floor = max(float(sigma11), 1e-300) * 2.0 ** -52
    return float(np.max(np.abs(np.asarray(sig) - truth) / np.maximum(truth, floor)))


def pass_algorithmic_bytes(m, n, b, cplx):
    """Bytes one Gram pass must move at least: A once (m n elements) and A W written once (m b)."""
    esz = 16 if cplx else 8
    return esz * (m * n + m * b)


def pass_tensor_flops(m, n, b):
    """Tensor-core work of one split-bf16 Gram pass: two products (A W and A^T (A W)), each over
    DIGIT_PAIRS digit pairs of 2 m n b multiply-adds (the unpadded block width b)."""
    return 2 * DIGIT_PAIRS * 2 * m * n * b


def pass_traffic(m, n):
    """DRAM bytes per Gram pass from the committed ncu summary of the split Gram kernels, scaled
    by m n from the bytes per element of A it states, if that summary was taken on the current
    gram_tc.cu (else None: the counters belong to another kernel)."""
    path = os.path.join(ROOT, "profiles", "gram_split_ncu_summary.md")
    src = os.path.join(ROOT, "paper_2602_16797_gb300", "csrc", "gram_tc.cu")
    try:
        txt = open(path).read()
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        tag, per = None, None
        for ln in txt.splitlines():
            if ln.startswith("gram_tc.cu sha256[:16]: "):
                tag = ln.split(": ", 1)[1].strip()
            if ln.startswith("dram bytes per element of A per pass: "):
                per = float(ln.split(": ", 1)[1].split()[0])
        return per * m * n if (tag == h and per is not None) else None
    except (OSError, ValueError):
        return None


def fp64_traffic(m, n):
    """DRAM bytes per FP64 Gram pass from the committed ncu summary of gram.cu, if current."""
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
        return per * m * n if (tag == h and per is not None) else None
    except (OSError, ValueError):
        return None


def gram_roofline(m, n, b, cplx, split, t_pass_s, peaks, fp64_peak_tf, fp64_peak_src):
    """Roofline object of the Gram pass (the dominant kernel pair) from its event-timed duration.

    Split path: the pass must move pass_algorithmic_bytes through HBM and run pass_tensor_flops
    on the tensor cores; the bound is whichever takes longer at its measured peak (HBM copy
    bandwidth; bf16 tensor throughput sustained, since the pass runs inside a long solve), and
    the other is reported beside it. FP64 path: 4 m n b (16 m n b complex) flops against the
    FP64 peak derived from the unit count and clock."""
    hbm = peaks.get("hbm_gbs") or 6800.0
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks.get("hbm_gbs") else "fallback 6.8 TB/s"
    tc = peaks.get("bf16_tflops_sustained") or 1700.0
    tc_src = ("MEASURED_PEAKS.json bf16_tflops_sustained (of measured)" if peaks.get("bf16_tflops_sustained")
              else "fallback 1.7 PFLOP/s sustained")
    by = pass_algorithmic_bytes(m, n, b, cplx)
    hbm_obj = {"bound": "hbm", "achieved": by / t_pass_s / 1e9, "peak": hbm, "unit": "GB/s",
               "frac": by / t_pass_s / 1e9 / hbm, "traffic": None, "bytes_per_pass": by,
               "peak_source": hbm_src}
    if not split:
        fl = (16.0 if cplx else 4.0) * m * n * b
        tf = fl / t_pass_s / 1e12
        hbm_obj["traffic"] = fp64_traffic(m, n)
        return {"bound": "alu", "achieved": tf, "peak": fp64_peak_tf, "unit": "TFLOP/s", "frac": tf / fp64_peak_tf,
                "traffic": hbm_obj["traffic"], "flops_per_pass": fl, "peak_source": fp64_peak_src,
                "kernel": "gram_kernel (fused A W, A^H A W), " + ("complex128" if cplx else "FP64"),
                "ms_per_pass": t_pass_s * 1e3, "hbm": hbm_obj}
    # complex A runs the real pass on its real view: m x 2n, block width 2b
    fl = pass_tensor_flops(m, 2 * n, 2 * b) if cplx else pass_tensor_flops(m, n, b)
    tc_obj = {"bound": "tensor", "achieved": fl / t_pass_s / 1e12, "peak": tc, "unit": "TFLOP/s",
              "frac": fl / t_pass_s / 1e12 / tc, "traffic": None, "flops_per_pass": fl, "peak_source": tc_src}
    hbm_obj["traffic"] = pass_traffic(m, 2 * n if cplx else n)
    t_hbm, t_tc = by / (hbm * 1e9), fl / (tc * 1e12)
    main, other = (tc_obj, hbm_obj) if t_tc > t_hbm else (hbm_obj, tc_obj)
    out = dict(main)
    out.update({"kernel": "split-bf16 Gram pass (gram_tc.cu: split of W, A W and A^T (A W) on tcgen05; A^T (A W) "
                          "on all SMs but those left to the TSQR merges and the Rayleigh-Ritz SVD beside it)"
                + ("; complex128 through its real view (gram_split_c.cu)" if cplx else ""),
                "ms_per_pass": t_pass_s * 1e3, "roof_ms": max(t_hbm, t_tc) * 1e3,
                "other": other})
    return out


# --------------------------------------------------------------------------------------- our arm

def _opts(rl, w, seed, prec, fixed_iters, gram):
    o = rl.rlobpcg_default_opts()
    o.d = w["d"]
    o.zeta = w["zeta"]
    o.sketch_prec = prec
    o.seed = seed
    o.gram_split = 1 if gram == "split" else 0
    if "stagnation" in w:
        o.use_stagnation = w["stagnation"]
    if "tau" in w:
        o.tau = w["tau"]
    if fixed_iters:
        o.fixed_iters = fixed_iters
    return o


def _timed_solves(rl, torch, plans, Ad, steps, stream, outs):
    """`steps` solves (matrix i % len, its seed's plan) between CUDA events on the plans' stream."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    infos = []
    torch.cuda.synchronize()
    ev[0].record(stream)
    for i in range(steps):
        info = rl.rlobpcg_info()
        rl.rlobpcg_solve(plans[i % len(plans)], Ad[i % len(Ad)].data_ptr(), Ad[i % len(Ad)].shape[1], -1.0,
                         *outs, info)
        ev[i + 1].record(stream)
        infos.append(info)
    torch.cuda.synchronize()
    lat = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    return ev[0].elapsed_time(ev[-1]), lat, infos


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2602_16797_gb300 import rlobpcg as rl

    w = WORKLOADS[args.workload]
    M, N, K, D = w["m"], w["n"], w["k"], w["d"]
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    rl.load()
    if "host" in w:
        hostA, truth = w["host"](M)
        Ad = [torch.from_numpy(A).to(dev) for A in hostA]
    else:
        Ad, truth = w["device"](M, dev)
        hostA = None
    dtype = rl.RLOBPCG_C128 if w["cplx"] else rl.RLOBPCG_F64
    tdt = torch.complex128 if w["cplx"] else torch.float64
    esz = 16 if w["cplx"] else 8
    stream = torch.cuda.current_stream(dev)
    split = args.gram == "split" and (2 * K if w["cplx"] else K) <= 24
    seeds = w["seeds"]
    # one plan per seed: a plan keeps the options it was made with (the seed of S among them)
    plans = [rl.rlobpcg_plan(M, N, K, dtype, _opts(rl, w, sd, w["prec"], args.fixed_iters, args.gram),
                             stream.cuda_stream) for sd in seeds]
    sigma = torch.empty(K, dtype=torch.float64, device=dev)
    resid = torch.empty(K, dtype=torch.float64, device=dev)
    V = torch.empty((N, K), dtype=tdt, device=dev)
    outs = (sigma.data_ptr(), V.data_ptr(), None, resid.data_ptr())

    for i in range(args.warmup):
        rl.rlobpcg_solve(plans[i % len(plans)], Ad[i % len(Ad)].data_ptr(), N, -1.0, *outs, rl.rlobpcg_info())
    torch.cuda.synchronize()
    replicas.barrier(world)
    clocks = ClockSampler(local_rank)
    clocks.start()
    ms_total, lat, infos = _timed_solves(rl, torch, plans, Ad, args.steps, stream, outs)
    clk = clocks.stop()
    replicas.barrier(world)
    ms_total = replicas.max_over_ranks(ms_total, world, device=dev)
    sig_last = sigma.cpu().numpy().copy()
    err_truth = sigma_err(sig_last, truth[(args.steps - 1) % len(truth)], infos[-1].sigma11)

    # mixed-precision form (FP32 sketch and R) on the same matrices, beside the plain form
    mixed = None
    if "mixed_prec" in w and not args.no_mixed:
        mplans = [rl.rlobpcg_plan(M, N, K, dtype, _opts(rl, w, sd, w["mixed_prec"], args.fixed_iters, args.gram),
                                  stream.cuda_stream) for sd in seeds]
        rl.rlobpcg_solve(mplans[0], Ad[0].data_ptr(), N, -1.0, *outs, rl.rlobpcg_info())
        msteps = max(2, args.steps // 3)
        mms, _, minfos = _timed_solves(rl, torch, mplans, Ad, msteps, stream, outs)
        ms_sig = sigma.cpu().numpy().copy()
        tr = truth[(msteps - 1) % len(truth)]
        mixed = {"sketch_prec": {1: "fp32", 2: "fp32 + fp64 refinement"}.get(w["mixed_prec"], "?"),
                 "solves_per_s": msteps / (mms * 1e-3), "ms_per_solve": mms / msteps, "steps": msteps,
                 "iters": [x.iters for x in minfos],
                 "per_iteration_ms": statistics.mean(x.ms_iterate / max(x.iters, 1) for x in minfos),
                 "phase_ms": {"sketch": statistics.mean(x.ms_sketch for x in minfos),
                              "factor": statistics.mean(x.ms_factor for x in minfos)},
                 "sigma_rel_err_vs_planted": sigma_err(ms_sig, tr, minfos[-1].sigma11)}
        for p in mplans:
            rl.rlobpcg_plan_destroy(p)

    # e2e: host buffers through the same C-ABI call (H2D of A and D2H of the results inside)
    pinned = [torch.from_numpy(A).pin_memory() for A in hostA] if hostA is not None else \
        [A.cpu().pin_memory() for A in Ad]
    sig_h = torch.empty(K, dtype=torch.float64).pin_memory()
    V_h = torch.empty((N, K), dtype=tdt).pin_memory()
    res_h = torch.empty(K, dtype=torch.float64).pin_memory()
    hout = (sig_h.data_ptr(), V_h.data_ptr(), None, res_h.data_ptr())
    e2e_steps = max(2, min(args.steps, 4))
    rl.rlobpcg_solve(plans[0], pinned[0].data_ptr(), N, -1.0, *hout, rl.rlobpcg_info())  # warm the host-A buffer
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        rl.rlobpcg_solve(plans[i % len(plans)], pinned[i % len(pinned)].data_ptr(), N, -1.0, *hout, rl.rlobpcg_info())
    e2e_s = time.perf_counter() - t0
    for p in plans:
        rl.rlobpcg_plan_destroy(p)

    gram_ms = sum(x.ms_gram for x in infos)
    passes = sum(x.gram_passes for x in infos)
    t_pass = gram_ms / max(passes, 1) * 1e-3
    props = torch.cuda.get_device_properties(dev)
    max_mhz = clk.get("sm_max_mhz") or 2070.0
    fp64_peak = props.multi_processor_count * FP64_UNITS_PER_SM_CLK * 2 * max_mhz * 1e6 / 1e12
    roofline = gram_roofline(M, N, K, w["cplx"], split, t_pass, measured_peaks(), fp64_peak,
                             f"derived: {props.multi_processor_count} SMs x {FP64_UNITS_PER_SM_CLK} DFMA/clk x 2 flop x "
                             f"{max_mhz:.0f} MHz")
    roofline["passes_timed"] = passes

    out = None
    if rank == 0:
        ms_per = ms_total / args.steps
        value = replicas.job_rate(args.steps, world, ms_total * 1e-3)
        iters = [x.iters for x in infos]
        result = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128" if w["cplx"] else "f64",
            "data": "synthetic (seeded; the paper's matrix families)",
            "config": {"workload": w["desc"], "m": M, "n": N, "k": K, "d": D, "zeta": w["zeta"],
                       "sketch": "fp32" if w["prec"] == 1 else "fp64", "matrices": w["matrices"],
                       "gram": ("split-bf16 tensor cores" + (" (real view of complex A)" if w["cplx"] else ""))
                               if split else ("fp64 CUDA cores" if not w["cplx"] else "complex128 CUDA cores"),
                       "fixed_iters": args.fixed_iters or None,
                       "l2": "input larger than L2; no flush" if M * N * esz > 129e6 else
                             "input smaller than L2 (each step is a full solve)",
                       "parallelism": f"replicas x{world}"},
            "per_iteration_ms": statistics.mean(x.ms_iterate / max(x.iters, 1) for x in infos),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "iters": iters, "stop_reasons": [x.stop_reason for x in infos],
            "sigma_rel_err_vs_planted": err_truth,
            "rr_sweeps_per_svd": round(sum(x.rr_sweeps for x in infos) / max(1, sum(x.rr_calls for x in infos)), 2),
            "phase_ms": {"sketch": statistics.mean(x.ms_sketch for x in infos),
                         "factor": statistics.mean(x.ms_factor for x in infos),
                         "iterate": statistics.mean(x.ms_iterate for x in infos),
                         "gram_per_pass": t_pass * 1e3,
                         "gram_ab_per_pass": sum(x.ms_gram_ab for x in infos) / max(passes, 1),
                         "gram_atb_per_pass": sum(x.ms_gram_atb for x in infos) / max(passes, 1),
                         "split_a": statistics.mean(x.ms_split_a for x in infos)},
            "sigma": [float(x) for x in sig_last],
            "roofline": roofline, "clocks": clk,
            "gpu_launches": int(sum(x.kernel_launches for x in infos)),
            "e2e": {"value": e2e_steps / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": esz * M * N,
                    "d2h_bytes_per_step": 8 * K + esz * N * K + 8 * K},
        }
        if mixed is not None:
            result["mixed"] = mixed
        if world == 1 and not args.no_cpu_baseline:
            t0 = time.perf_counter()
            ph = oracle_sample_phases(w, run_to_stop=True)
            secs = time.perf_counter() - t0
            gi = statistics.mean(iters)
            est = oracle_full_solve_seconds(w, ph, gi)
            result["cpu_baseline"] = {
                "value": 1.0 / est, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                "sample": (f"oracle (numpy/LAPACK, all host cores) on a {ph['sample_m']}-row sample of the same matrix "
                           f"family ({secs:.1f} s): one run to its own stop ({ph['stop_iters']} iterations) and one "
                           f"with 1 iteration give {ph['t_iter']:.3f} s per iteration and {ph['t_once_stream']:.2f} s "
                           f"of one-time work that streams A (both x {M / ph['sample_m']:g} for m = {M}), plus the "
                           f"SVD of the d x n sketch ({ph['t_svd']:.2f} s, size-independent), at the GPU's "
                           f"{gi:g} iterations"),
                "oracle_iters_on_sample": ph["stop_iters"], "gpu_iters": gi,
                "per_iteration_s_full_size": ph["t_iter"] * M / ph["sample_m"]}
            one = oracle_rate_one_thread(args.workload, int(round(gi)))
            if one is not None:
                result["cpu_baseline"]["value_1_thread"] = one[0]
                result["cpu_baseline"]["sample"] += (f"; value_1_thread: the same estimate from a 1- and 3-iteration "
                                                     f"sample with every BLAS pool at one thread ({one[1]:.1f} s)")
        out = result
    return out


def run_reference(args, rank, world):
    """The CPU oracle, as it stands, on the host cores: each step times it per phase on a row sample
    of the workload and scales it to the full size at the iteration count the oracle's own
    stopping rule reaches on that sample (measured once, before the timed steps)."""
    if rank != 0:
        return None
    w = WORKLOADS[args.workload]
    ms = w.get("ref_sample_m", w["sample_m"])
    ph0 = oracle_sample_phases(w, run_to_stop=True, sample_m=ms)
    iters = ph0["stop_iters"]
    per = []
    for i in range(args.warmup + args.steps):
        ph = oracle_sample_phases(w, run_to_stop=False, sample_m=ms)
        if i >= args.warmup:
            per.append(oracle_full_solve_seconds(w, ph, iters))
    total = sum(per)
    v = args.steps / total
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128" if w["cplx"] else "f64", "data": "synthetic (seeded; the paper's matrix families)",
            "config": {"workload": w["desc"], "m": w["m"], "n": w["n"], "k": w["k"], "d": w["d"], "zeta": w["zeta"],
                       "parallelism": "cpu oracle, rank 0 only"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"each step: the oracle on a {ph0['sample_m']}-row sample of the same matrix "
                                       f"family, 1 and 3 fixed iterations, scaled to m = {w['m']} (the parts that stream "
                                       f"A) at the {iters} iterations its stopping rule takes on the sample"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_block_study(args, rank, world, local_rank):
    """Block sizes b in {1, 3, 5, 10, 20} on the clustered 1e6 x 2000 matrix of Sec. 4.2 (16 GB
    FP64, Haar U and V, sigma_i = exp(-log(1e10) ((i-1)/(n-1))^(1/256))), one triplet (k = 1)
    wanted: per block size the iterations, matrix-vector products (b per iteration), device
    time of the solve, the relative error of the smallest singular value against the planted one
    and the sine of the angle of its vector to the planted one, and the per-iteration relative
    error of the smallest Ritz value. Every block size runs the Gram products on the tensor
    cores (split-bf16 digits, b <= 24)."""
    import torch

    from paper_2602_16797_gb300 import rlobpcg as rl
    from paper_2602_16797_gb300 import workloads as wl
    if rank != 0:
        return None
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    rl.load()
    m, n = args.study_m, args.study_n
    A, s_true, V_true = wl.clustered_large_device(m=m, n=n, device=dev)
    smin, vmin = s_true[-1], V_true[:, -1]
    gap = (s_true[-2] ** 2 - s_true[-1] ** 2) / s_true[-1] ** 2
    stream = torch.cuda.current_stream(dev)
    sigma = torch.empty(1, dtype=torch.float64, device=dev)
    resid = torch.empty(1, dtype=torch.float64, device=dev)
    V = torch.empty((n, 1), dtype=torch.float64, device=dev)
    rows = []
    blocks = [int(x) for x in args.blocks.split(",")]
    for i, b in enumerate(blocks):
        o = rl.rlobpcg_default_opts()
        o.seed = 1006
        o.block = b
        o.max_iter = args.study_max_iter
        plan = rl.rlobpcg_plan(m, n, 1, rl.RLOBPCG_F64, o, stream.cuda_stream)
        if i == 0:
            rl.rlobpcg_solve(plan, A.data_ptr(), n, -1.0, sigma.data_ptr(), V.data_ptr(), None, resid.data_ptr(),
                             rl.rlobpcg_info())   # warm-up (kernels, clocks)
        info = rl.rlobpcg_info()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        rl.rlobpcg_solve(plan, A.data_ptr(), n, -1.0, sigma.data_ptr(), V.data_ptr(), None, resid.data_ptr(), info)
        e1.record(stream)
        torch.cuda.synchronize()
        th, rs = rl.rlobpcg_history(plan)
        rl.rlobpcg_plan_destroy(plan)
        v = V.cpu().numpy()[:, 0]
        sin = float(np.sqrt(max(0.0, 1.0 - abs(float(v @ vmin)) ** 2)))
        err_hist = [float(abs(t - smin) / smin) for t in th[:, -1]]
        ms_it = info.ms_iterate / max(info.iters, 1)
        once = info.ms_sketch + info.ms_factor + info.ms_split_a
        # cost to first reach each relative sigma error: iterations, matvecs (b per iteration plus
        # the start block), device time (one-time part + iterations at the measured rate)
        reach = {}
        for thr in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8):
            it = next((t for t, e in enumerate(err_hist) if e <= thr), None)
            reach[f"{thr:g}"] = None if it is None else {"iters": it, "matvecs": b * (it + 1),
                                                         "ms": once + it * ms_it}
        rows.append({"b": b, "gram": "split-bf16 tensor cores" if b <= 24 else "fp64 CUDA cores",
                     "iters": info.iters, "matvecs": info.matvecs, "stop_reason": info.stop_reason,
                     "ms": e0.elapsed_time(e1), "ms_per_iteration": ms_it, "ms_one_time": once,
                     "sigma_rel_err": float(abs(sigma.item() - smin) / smin), "vector_sin_angle": sin,
                     "reach": reach, "sigma_rel_err_history": err_hist})
    return {"metric": "block-size study (Sec. 4.2): iterations, matvecs, wall-clock and accuracy per block size",
            "value": None, "unit": None, "n_gpus": 1, "dtype": "f64", "data": "synthetic (seeded; Sec. 4.2 recipe)",
            "config": {"workload": f"clustered m={m} n={n} k=1, sigma_i = exp(-log(1e10) ((i-1)/(n-1))^(1/256))",
                       "d": 4 * n, "zeta": 8, "gap_rel": float(gap), "sigma_min": float(smin)},
            "blocks": rows}


def run_serve(args, rank, world, local_rank):
    """Serving stream: `--requests` requests (half Loewner, half planted; m log-uniform in
    [2e3, 5e5], n uniform in [20, 400], k in {1, 2, 4}) under an HBM admission budget of 150 GB,
    drawn from a pool of `--pool` seeded matrices in pinned host memory (request r: pool entry
    r mod pool, its own sketch seed). Measures the saturated rate of the batched server (`--slots`
    workers; the iterations of every admitted request with m n b <= 2^23 in one batch engine,
    larger ones whole with their Gram products on the tensor cores), the same stream on the
    per-stream server (`--stream-slots` whole solves overlapping) and one solve at a time, and
    Poisson arrivals at 0.5 / 0.9 / 1.2 x the batched saturated rate (p50 / p99 latency from
    submit to result, host copy of A included)."""
    import torch

    from paper_2602_16797_gb300 import rlobpcg as rl
    from paper_2602_16797_gb300 import workloads as wl
    if rank != 0:
        return None
    torch.cuda.set_device(local_rank)
    rl.load()
    t_gen = time.perf_counter()
    pool = wl.serve_pool(args.pool)
    t_gen = time.perf_counter() - t_gen
    reqs = []
    for r in range(args.requests):
        A, k, kind = pool[r % len(pool)]
        reqs.append((A, k, wl.SERVE_SEED_BASE + r))
    budget = 150 * (1 << 30)

    def opts(seed):
        o = rl.rlobpcg_default_opts()   # whole solves: Gram products on the tensor cores
        o.seed = seed
        return o

    def stream(slots, mode, arrivals=None):
        srv = rl.rlobpcg_server_create(budget, slots, local_rank, mode)
        t0 = time.perf_counter()
        tickets = []
        for i, (A, k, seed) in enumerate(reqs):
            if arrivals is not None:
                dt = t0 + arrivals[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            tickets.append(rl.rlobpcg_server_submit(srv, A.data_ptr(), A.shape[0], A.shape[1], A.shape[1], k,
                                                    rl.RLOBPCG_F64, opts(seed)))
        iters = []
        for (A, k, seed), t in zip(reqs, tickets):
            info = rl.rlobpcg_info()
            rl.rlobpcg_server_wait(srv, t, None, None, None, info)
            iters.append(info.iters)
        makespan = time.perf_counter() - t0
        st = rl.rlobpcg_server_stats(srv)
        st["engine"] = rl.rlobpcg_server_engine_stats(srv)
        rl.rlobpcg_server_destroy(srv)
        st["makespan_s"] = makespan
        st["rate"] = len(reqs) / makespan
        st["mean_iters"] = float(np.mean(iters))
        return st

    # warm-up: the batched kernels' tile shapes for every class of the pool, then a short stream
    for A, k, seed in reqs[:len(pool)]:
        rl.rlobpcg_batch_tile(A.shape[1], k)
    B, S = rl.RLOBPCG_SERVE_BATCHED, rl.RLOBPCG_SERVE_STREAMS
    sat = stream(args.slots, B)
    per_stream = stream(args.stream_slots, S)
    seq = stream(1, S)
    lat = {}
    rng = np.random.default_rng(4242)
    for f in (0.5, 0.9, 1.2):
        lam = f * sat["rate"]
        arr = np.cumsum(rng.exponential(1.0 / lam, len(reqs)))
        st = stream(args.slots, B, arr)
        lat[f"{f}x"] = {"offered_per_s": lam, "solves_per_s": st["rate"], "p50_ms": st["p50_ms"],
                        "p99_ms": st["p99_ms"], "peak_running": st["peak_running"], "peak_gb": st["peak_bytes"] / 1e9}
    bytes_in = float(np.mean([A.numel() * 8 for A, _, _ in reqs]))
    return {"metric": METRIC, "value": sat["rate"], "unit": "solves/s", "n_gpus": 1, "steps": len(reqs),
            "warmup": len(pool), "ms_per_step": 1e3 / sat["rate"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded; the paper's matrix families)",
            "config": {"workload": f"serving stream of {len(reqs)} requests over a pool of {len(pool)} matrices "
                                   f"(half Loewner, half planted; m log-uniform [2e3,5e5], n U[20,400], k in "
                                   f"{{1,2,4}}), HBM budget 150 GB, batched server with {args.slots} slots",
                       "parallelism": "continuous batching on one GPU", "pool_generation_s": t_gen},
            "batched": {"solves_per_s": sat["rate"], "p50_ms": sat["p50_ms"], "p99_ms": sat["p99_ms"],
                        "peak_running": sat["peak_running"], "mean_iters": sat["mean_iters"],
                        "engine": sat["engine"]},
            "per_stream": {"slots": args.stream_slots, "solves_per_s": per_stream["rate"],
                           "p50_ms": per_stream["p50_ms"], "p99_ms": per_stream["p99_ms"],
                           "mean_iters": per_stream["mean_iters"]},
            "one_at_a_time": {"solves_per_s": seq["rate"], "p50_ms": seq["p50_ms"], "p99_ms": seq["p99_ms"]},
            "poisson_batched": lat,
            "e2e": {"value": sat["rate"], "unit": "solves/s", "h2d_bytes_per_step": bytes_in,
                    "d2h_bytes_per_step": None}}


def run_fig1(args, rank, world, local_rank):
    """Sec. 1.1's comparison (Fig. 1) on the GPU: the easy and hard m x n problems (default
    2e6 x 4e3, 64 GB FP64 each), the smallest singular triplet (b = k = 1) by RLOBPCG and by the
    same LOBPCG with the diagonal preconditioner and with none, all from the sketch-and-solve
    start v0 and with the paper's iteration cap (200 for b = 1). Reported per method: the relative
    error (theta_t - sigma_n) / sigma_n of the estimate after every iteration (theta_t = ||A v_t||
    for the Ritz vector), the one-time and per-iteration device times, and the time to reach the
    best error RLOBPCG reaches. Gram products on the tensor cores (split-bf16: A 64 GB + its byte
    digits 128 GB on the device)."""
    import torch

    from paper_2602_16797_gb300 import rlobpcg as rl
    from paper_2602_16797_gb300 import workloads as wl
    if rank != 0:
        return None
    torch.cuda.set_device(local_rank)
    rl.load()
    m, n = args.fig1_m, args.fig1_n
    # (name, preconditioner, sketch precision): the three methods of Sec. 1.1, and RLOBPCG with its
    # factor in FP32 refined once in FP64 (the mixed-precision form)
    variants = [("rlobpcg", rl.RLOBPCG_PRECOND_SKETCH, rl.RLOBPCG_SKETCH_F64),
                ("rlobpcg_f32_refined", rl.RLOBPCG_PRECOND_SKETCH, rl.RLOBPCG_SKETCH_F32_REFINE),
                ("lobpcg_diag", rl.RLOBPCG_PRECOND_DIAG, rl.RLOBPCG_SKETCH_F64),
                ("lobpcg_none", rl.RLOBPCG_PRECOND_NONE, rl.RLOBPCG_SKETCH_F64)]
    out = {}
    t_gen = time.perf_counter()
    for kind, A, sigma in wl.fig1_device(m, n):
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t_gen
        sn = float(sigma[-1])
        res = {"sigma_n": sn, "generation_s": gen_s}
        for name, pc, prec in variants:
            o = rl.rlobpcg_default_opts()
            o.seed = 7
            o.block = 1
            o.precond = pc
            o.sketch_prec = prec
            st = torch.cuda.current_stream().cuda_stream
            plan = rl.rlobpcg_plan(m, n, 1, rl.RLOBPCG_F64, o, st)
            sig = torch.empty(1, dtype=torch.float64, device="cuda")
            V = torch.empty((n, 1), dtype=torch.float64, device="cuda")
            info = rl.rlobpcg_info()
            try:
                rc = rl.rlobpcg_solve(plan, A.data_ptr(), n, -1.0, sig.data_ptr(), V.data_ptr(), None, None, info)
                th, rs = rl.rlobpcg_history(plan)
            finally:
                rl.rlobpcg_plan_destroy(plan)
            err = (th[:, -1] - sn) / sn
            per_it = info.ms_iterate / max(1, info.iters)
            setup = info.ms_sketch + info.ms_factor
            res[name] = {"status": rc, "iters": info.iters, "stop_reason": info.stop_reason,
                         "setup_ms": setup, "sketch_ms": info.ms_sketch, "factor_ms": info.ms_factor,
                         "ms_per_iteration": per_it, "ms_total": info.ms_total,
                         "rel_err_v0": float(err[0]), "rel_err_final": float(err[-1]),
                         "rel_err_every_10": [float(x) for x in err[::10]]}
        best = res["rlobpcg"]["rel_err_final"]
        for name, _, _ in variants:
            r = res[name]
            errs = r["rel_err_every_10"]
            hit = next((i * 10 for i, e in enumerate(errs) if e <= max(best, 0) * 1.0001 + 1e-300), None)
            r["ms_to_rlobpcg_best"] = (r["setup_ms"] + hit * r["ms_per_iteration"]) if hit is not None else None
        out[kind] = res
        t_gen = time.perf_counter()
    return {"metric": "Fig. 1 (Sec. 1.1): relative error of the smallest singular value vs time", "unit": "ms",
            "config": {"workload": f"Sec. 1.1 easy and hard problems, m={m} n={n}, b=k=1, split-bf16 Gram",
                       "data": "synthetic (Haar U from a GPU QR; the paper's V and sigma recipes)"},
            "results": out}


def run_batch_small(args, rank, world, local_rank):
    """Many small solves at once: `--batch-count` planted matrices (m log-uniform in [2e3, 1e5],
    n uniform in [20, 400], k in {1, 2, 4}; sigma logspace(0,-6) with the k smallest logspace(-10,-9))
    on the device, solved by rlobpcg_solve_batch (set-ups on their plan streams, iterations of all
    solves together in the batch engine) and, as the baseline, by rlobpcg_solve one at a time.
    Timed: `--steps` batches after `--warmup` (the first also tunes the tile shapes)."""
    import torch

    from paper_2602_16797_gb300 import rlobpcg as rl
    from paper_2602_16797_gb300 import workloads as wl
    if rank != 0:
        return None
    torch.cuda.set_device(local_rank)
    rl.load()
    if args.batch_tile:   # pin every class's tile shape (e.g. to profile without the autotuner's launches)
        tr, rt = (int(x) for x in args.batch_tile.split(":"))
        for nc in (32, 64, 128, 256, 512):
            for b in (1, 2, 4):
                rl.rlobpcg_batch_set_tile(nc, b, tr, rt)
    rng = np.random.default_rng(3)
    mats, ks = [], []
    for r in range(args.batch_count):
        m = int(np.exp(rng.uniform(np.log(2e3), np.log(1e5))))
        n = int(rng.integers(20, 401))
        k = int(rng.choice([1, 2, 4]))
        m = max(m, 4 * n)
        sigma = np.concatenate([np.logspace(0, -6, n - k), np.logspace(-10, -9, k)])
        mats.append(wl.planted_on_device(50000 + r, m, sigma)[0])
        ks.append(k)
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(8)]

    def opts(k):
        o = rl.rlobpcg_default_opts()
        o.seed = 1
        o.block = k
        o.gram_split = 0
        return o

    def batch():
        plans = [rl.rlobpcg_plan(A.shape[0], A.shape[1], k, rl.RLOBPCG_F64, opts(k), streams[i % 8].cuda_stream)
                 for i, (A, k) in enumerate(zip(mats, ks))]
        outs = [(torch.empty(k, dtype=torch.float64, device="cuda"),
                 torch.empty((A.shape[1], k), dtype=torch.float64, device="cuda")) for A, k in zip(mats, ks)]
        torch.cuda.synchronize()
        t = time.perf_counter()
        rc, infos, st = rl.rlobpcg_solve_batch(plans, [A.data_ptr() for A in mats], [A.shape[1] for A in mats],
                                              [o[0].data_ptr() for o in outs], [o[1].data_ptr() for o in outs],
                                              None, None, 0)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        for p in plans:
            rl.rlobpcg_plan_destroy(p)
        return dt, infos

    for _ in range(args.warmup):
        batch()
    times, iters = [], []
    for _ in range(args.steps):
        dt, infos = batch()
        times.append(dt)
        iters.append(float(np.mean([i.iters for i in infos])))
    t = time.perf_counter()
    seq_iters = []
    for A, k in zip(mats, ks):
        sig, V, U, res, info = rl.solve(A, k, opts=opts(k))
        seq_iters.append(info["iters"])
    torch.cuda.synchronize()
    seq = time.perf_counter() - t
    dt = float(np.median(times))
    return {"metric": "solves/s of many small solves (batched iterations)", "value": len(mats) / dt,
            "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic (seeded planted spectra)",
            "config": {"workload": f"{len(mats)} small solves (m log-uniform [2e3,1e5], n U[20,400], k in {{1,2,4}})",
                       "parallelism": "batch engine on one GPU"},
            "mean_iters": float(np.mean(iters)), "one_at_a_time": {"solves_per_s": len(mats) / seq,
                                                                   "mean_iters": float(np.mean(seq_iters))}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["serve_stream", "block_study", "fig1", "batch_small"],
                    default=DEFAULT_WORKLOAD)
    ap.add_argument("--batch-count", type=int, default=64, help="batch_small: solves per batch")
    ap.add_argument("--batch-tile", default="", help="batch_small: pin every class's tile shape, trows:rt")
    ap.add_argument("--fig1-m", type=int, default=2_000_000, help="fig1: rows")
    ap.add_argument("--fig1-n", type=int, default=4000, help="fig1: columns")
    ap.add_argument("--blocks", default="1,3,5,10,20", help="block_study: block sizes")
    ap.add_argument("--study-m", type=int, default=1_000_000, help="block_study: rows")
    ap.add_argument("--study-n", type=int, default=2000, help="block_study: columns")
    ap.add_argument("--study-max-iter", type=int, default=0,
                    help="block_study: iteration cap (0: the paper's, 200 for b = 1 and 100 otherwise)")
    ap.add_argument("--gram", choices=["split", "fp64"], default="split",
                    help="Gram products: split-bf16 on the tensor cores (default) or FP64 CUDA cores")
    ap.add_argument("--fixed-iters", type=int, default=0,
                    help="run exactly this many LOBPCG iterations per solve (no stop test)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision form beside the plain one")
    ap.add_argument("--requests", type=int, default=2000, help="serve_stream: number of requests")
    ap.add_argument("--slots", type=int, default=64, help="serve_stream: solves iterating together (batched server)")
    ap.add_argument("--stream-slots", type=int, default=8, help="serve_stream: whole solves overlapping (per-stream server)")
    ap.add_argument("--pool", type=int, default=48, help="serve_stream: distinct matrices the requests are drawn from")
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
    elif args.workload == "block_study":
        out = run_block_study(args, rank, world, local_rank)
    elif args.workload == "fig1":
        out = run_fig1(args, rank, world, local_rank)
    elif args.workload == "batch_small":
        out = run_batch_small(args, rank, world, local_rank)
    else:
        out = run_ours(args, rank, world, local_rank)
    replicas.finish(world)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
