#!/usr/bin/env python
"""Benchmark of the AM sparse-PCA hot path on GB300.

A step is one pass of the whole path over one batch: for each of the 8 formulations of
Table 1, one solve of Algorithm 2 from r = 1024 unit-norm starts (start normalisation, sweeps
until every start has stopped, FP64 objective, best start) on the spiked-model workload
  A = sum_{k=1..5} theta_k u_k v_k^T + N(0,1),  n = 5000, p = 20000 (FP32, 400 MB > L2),
  theta_k = (40, 30, 20, 15, 10) sqrt(n / p), u_k Gaussian unit, v_k unit with 50 nonzeros,
  s = 50 (L0), sqrt(50) (L1 radius), gamma by the Section 4.1 rule targeting 50 nonzeros for
  the first 10 sweeps (penalty forms), at most 100 sweeps, tol 1e-9.

Metric: AM sweeps x starts per second (the sum over solves of the sweeps each start ran),
with solves/s and the p50/p99 latency of single solves.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]
  python bench.py --scan paper-shapes|text-corpus|few-starts|precision|many-problems|serving|economies
  python bench.py --tune   (the grouped contraction's tile shapes: writes paper_1212_4137_gb300/grouped_tiles.json)
(the scans print one JSON line per case; the clocks sampled during a run go to SPCA_CLOCKS_DIR,
else the temporary directory)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "AM sweeps·starts/s and solves/s (p50/p99) at ≤1e-3 rel. obj. error vs plain FP32"
UNIT = "sweeps*starts/s"

WORKLOADS = {
    # the spiked-model workload (all 8 formulations, r = 1024)
    "spiked-5000x20000-r1024": dict(n=5000, p=20000, r=1024, spikes=(40.0, 30.0, 20.0, 15.0, 10.0),
                                    nnz=50, s=50, forms=(1, 2, 3, 4, 5, 6, 7, 8), max_iter=100,
                                    tol=1e-9, calib=10, data_seed=7, start_seed=8),
    # the small dense case (n = 100, p = 500, N(0,1), form 1, s = 10, r = 16)
    "gaussian-100x500-r16": dict(n=100, p=500, r=16, spikes=None, nnz=0, s=10, forms=(1,),
                                 max_iter=100, tol=1e-9, calib=10, data_seed=1, start_seed=2),
}
DEFAULT_WORKLOAD = "spiked-5000x20000-r1024"

# DRAM traffic of one v = A^T y launch of the tensor-core contraction at the spiked workload's size
# with 1024 active starts (dram__bytes_read.sum + dram__bytes_write.sum of an ncu capture: 473.5 MB
# + 83.0 MB), and the algorithmic bytes of that launch: two FP16 planes of A^T (400 MB), two of Y
# (20.5 MB), V written once (81.9 MB)
V_TRAFFIC_BYTES = 556.5e6
V_ALG_BYTES = 502.4e6

# peak of the FP32 CUDA-core pipe: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.070 GHz
SIMT_FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


_INPUTS = {}


def make_inputs(w):
    key = (w["n"], w["p"], w["data_seed"])
    if key not in _INPUTS:
        _INPUTS[key] = _make_inputs(w)
    return _INPUTS[key]


def _make_inputs(w):
    from paper_1212_4137_gb300 import inputs as I
    n, p = w["n"], w["p"]
    if w["spikes"] is None:
        A = I.gaussian_matrix(n, p, w["data_seed"]).astype(np.float32)
    else:
        A = I.spiked_matrix(n, p, I.spiked_thetas(n, p, w["spikes"]), w["nnz"], w["data_seed"],
                            dtype=np.float32)
    return A


def solve_kwargs(w, form):
    if form in (1, 2, 3, 4):
        return dict(s=float(w["s"]))
    return dict(s=float(w["s"]), gamma_target=True, calib=w["calib"])


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        # the samples' file: SPCA_CLOCKS_DIR, else the system's temporary directory
        out_dir = os.environ.get("SPCA_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"spca_clocks_rank{device_index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        med = statistics.median(sm) if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------- our arm
def run_ours(args, w, rank, world, local_rank):
    import torch

    from paper_1212_4137_gb300 import build, spca
    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)

    A = make_inputs(w)
    n, p, r = w["n"], w["p"], w["r"]
    from paper_1212_4137_gb300 import inputs as I
    G = I.raw_starts(p, r, w["start_seed"] + 1000 * rank).astype(np.float32)   # weak scaling: own starts
    Ad = torch.from_numpy(A).to(dev)
    Gd = torch.from_numpy(G).to(dev)
    torch.cuda.synchronize(dev)
    h = spca.Handle(Ad, stream=stream.cuda_stream)

    vstats = {"launches": 0, "ms": 0.0, "tensor_flop": 0.0, "method_flop": 0.0}

    def one_step(times=None):
        sw = 0
        for form in w["forms"]:
            t0 = time.perf_counter()
            if times is not None:
                l0, m0 = h.profile_query(spca.SPCA_K_V)
            out = h.solve(form, r, max_iter=w["max_iter"], tol=w["tol"], x0=Gd.data_ptr(), x0_device=True,
                          **solve_kwargs(w, form))
            if times is not None:
                times.append(time.perf_counter() - t0)
                l1, m1 = h.profile_query(spca.SPCA_K_V)
                # algorithmic tensor-pipe flops of v = A^T y: each sweep of each active start
                # contracts one column with 2 (L1 variance, y = +-1) or 3 (L2 variance) FP16
                # plane products (frozen starts are not contracted)
                vstats["launches"] += l1 - l0
                vstats["ms"] += m1 - m0
                vstats["tensor_flop"] += out["sweeps_total"] * 2.0 * n * p * (2 if form % 2 == 0 else 3)
                vstats["method_flop"] += out["sweeps_total"] * 2.0 * n * p
            sw += out["sweeps_total"]
        return sw

    for _ in range(args.warmup):
        one_step()
    barrier(world)
    # inside the timed region only the dominant kernel (v = A^T y) is bracketed by events
    h.profile(True, kernels=(spca.SPCA_K_V,))
    lat = []
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize(dev)
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sweeps = 0
        for _ in range(args.steps):
            sweeps += one_step(lat)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
    ms = e0.elapsed_time(e1)
    launches, _ = h.profile_query(spca.SPCA_K_ALL)
    h.profile(False)
    clocks = clk.summary()
    # per-kernel shares of device time from one more (untimed) step with every launch timed
    h.profile(True)
    sweeps_one = one_step()   # (the sweeps of this step: the per-kernel times below are this step's)
    kern = {}
    for kid, name in spca.KERNEL_NAMES.items():
        kern[name] = h.profile_query(kid)
    h.profile(False)

    ms_max = reduce_max(ms, world)
    sweeps_all = reduce_sum(sweeps, world)
    solves_all = reduce_sum(len(lat), world)
    value = sweeps_all / (ms_max / 1e3)

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e_steps = 0 if args.no_e2e else args.steps   # the same number of steps as the device-timed value
    if e2e_steps:
        A_pin = torch.from_numpy(A).pin_memory()
        G_pin = torch.from_numpy(G).pin_memory()
    barrier(world)
    t0 = time.perf_counter()
    e2e_sweeps = 0
    d2h = 0
    for _ in range(e2e_steps):
        h2 = spca.Handle(A_pin.numpy(), stream=stream.cuda_stream)
        for form in w["forms"]:
            out = h2.solve(form, r, max_iter=w["max_iter"], tol=w["tol"], x0=G_pin.numpy(),
                           **solve_kwargs(w, form))
            e2e_sweeps += out["sweeps_total"]
            d2h += 4 * (p + n) + 8 * int(out["nnz"]) + 64
        h2.close()
    torch.cuda.synchronize(dev)
    e2e_s = reduce_max(time.perf_counter() - t0, world)
    e2e_value = reduce_sum(e2e_sweeps, world) / e2e_s if e2e_steps else 0.0
    h2d = A.nbytes + len(w["forms"]) * G.nbytes
    h.close()

    if rank != 0:
        return None
    # roofline of the dominant kernel (largest share of device time)
    shares = {k: v[1] for k, v in kern.items()}
    total_ms = sum(shares.values()) or 1.0
    dom = max(shares, key=shares.get)
    peaks = load_peaks()
    roof = None
    if dom == "v" and vstats["ms"] > 0:
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        # the method's work (2 n p flop per sweep*start: every entry of v = A^T y of every active
        # start) over the measured launch time of v; the executed plane products beside it
        method = vstats["method_flop"] / (vstats["ms"] / 1e3) / 1e12
        executed = vstats["tensor_flop"] / (vstats["ms"] / 1e3) / 1e12
        roof = {"kernel": "v = A^T y (k_gemm_tc2: tcgen05 on FP16 planes, FP32 accumulate)", "bound": "tensor",
                "achieved": round(method, 1), "peak": peak, "unit": "TFLOP/s",
                "frac": round(method / peak, 4),
                "per_unit": "2*n*p flop per sweep*start (active starts only): the algorithmic work of v = A^T y",
                "units_per_launch": "the active starts of one sweep",
                "executed_plane_tflops": round(executed, 1), "executed_plane_frac": round(executed / peak, 4),
                "executed_per_unit": "2*n*p*(2 plane products for L1 variance, 3 for L2 variance) FP16 flop",
                # DRAM read + write of one launch from an ncu capture of this kernel (the first
                # v = A^T y of formulation 1: N = 1024 active starts, three plane products),
                # against its algorithmic bytes (A planes once, Y planes, V written once)
                "traffic": V_TRAFFIC_BYTES, "traffic_note": "bytes per launch, N = 1024 launch (ncu)",
                "algorithmic_bytes_same_launch": V_ALG_BYTES,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured; FP16 and BF16 dense rates are equal)",
                "launches": vstats["launches"], "avg_launch_ms": round(vstats["ms"] / max(1, vstats["launches"]), 4)}
    elif dom == "xstep" and kern["xstep"][1] > 0 and kern["v"][0] == 0:
        # a small problem: every sweep of every start in one launch (k_small_sweeps, charged to the
        # x-step's timer); its work is the two products on the CUDA cores, 4 n p flop per sweep*start
        achieved = 4.0 * n * p * sweeps_one / (kern["xstep"][1] / 1e3) / 1e12
        roof = {"kernel": "every sweep of a start in one launch (k_small_sweeps: u = A x, v = A^T y, y-step, x-step)",
                "bound": "alu", "achieved": round(achieved, 4), "peak": round(SIMT_FP32_PEAK_TFLOPS, 1),
                "unit": "TFLOP/s", "frac": round(achieved / SIMT_FP32_PEAK_TFLOPS, 5), "traffic": None,
                "per_unit": "4*n*p flop per sweep*start (the two products, FP32 FMA)",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (derived)",
                "launches": kern["xstep"][0]}
    elif dom == "xstep" and kern["xstep"][1] > 0:
        achieved = 8.0 * p * sweeps_one / (kern["xstep"][1] / 1e3) / 1e9
        roof = {"kernel": "x-step (k_xstep)", "bound": "hbm", "achieved": round(achieved, 1),
                "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                "frac": round(achieved / peaks.get("hbm_gbs", 6701.5), 4), "traffic": None,
                "per_launch": "8*p bytes per active start (read v, write x)", "launches": kern["xstep"][0]}
    lat_ms = sorted(1e3 * t for t in lat)
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args, w, world),
        "solves_per_s": round(solves_all / (ms_max / 1e3), 3),
        "solve_latency_ms": {"p50": round(float(np.percentile(lat_ms, 50)), 3),
                             "p99": round(float(np.percentile(lat_ms, 99)), 3)},
        "sweeps_starts": int(sweeps_all),
        "kernels_ms_share": {k: round(v / total_ms, 4) for k, v in shares.items()},
        "roofline": roof,
        "e2e": ({"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                 "d2h_bytes_per_step": int(d2h // e2e_steps), "steps": e2e_steps} if e2e_steps else None),
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    return line


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "fallback": True}


# ---------------------------------------------------------------------------- CPU baseline
def oracle_sample(w, A64, G, form, starts, sweeps):
    from oracle import oracle
    kw = solve_kwargs(w, form)
    kw.pop("calib", None)
    t0 = time.perf_counter()
    res = oracle.solve(A64, form, G[:starts].astype(np.float64), max_iter=sweeps, tol=-1,
                       calib=w["calib"], **kw)
    dt = time.perf_counter() - t0
    return int(res.iters.sum()), dt, oracle.num_threads()


def cpu_baseline(w, A, G, starts=32, sweeps=10):
    A64 = A.astype(np.float64)
    sw, dt, cores = oracle_sample(w, A64, G, 1, starts, sweeps)
    return {"value": round(sw / dt, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"formulation 1, first {starts} of the {w['r']} starts, {sweeps} sweeps each "
                      f"({sw} sweeps*starts in {dt:.1f} s), FP64, OpenMP over starts"}


def workload_config(args, w, world):
    """The `config` object of the benchmark line (the same for both arms)."""
    a_bytes = w["n"] * w["p"] * 4
    l2 = ("inputs larger than L2 (A = %d MB)" % (a_bytes // 2**20) if a_bytes > 129 * 2**20
          else "A = %.1f MB stays in L2, not flushed: a resident problem's solve latency" % (a_bytes / 2**20))
    return {"workload": args.workload, "n": w["n"], "p": w["p"], "r": w["r"], "formulations": list(w["forms"]),
            "s": w["s"], "gamma_mode": "target_nnz (Section 4.1), %d calibration sweeps" % w["calib"],
            "max_iter": w["max_iter"], "tol": w["tol"], "storage": "fp32", "engine": "auto", "l2": l2,
            "parallelism": f"replicas x{world} (starts sharded, no collective)"}


def run_reference(args, w, rank, world):
    if rank != 0:
        return None
    from oracle import oracle
    oracle.build()
    from paper_1212_4137_gb300 import inputs as I
    A = make_inputs(w)
    A64 = A.astype(np.float64)
    G = I.raw_starts(w["p"], w["r"], w["start_seed"]).astype(np.float32)
    starts, sweeps = (16, 5) if w["n"] * w["p"] > 1e7 else (w["r"], w["max_iter"])
    forms = w["forms"]
    for k in range(args.warmup):
        oracle_sample(w, A64, G, forms[k % len(forms)], starts, sweeps)
    tot_sw, tot_dt, cores = 0, 0.0, 1
    for k in range(args.steps):
        sw, dt, cores = oracle_sample(w, A64, G, forms[k % len(forms)], starts, sweeps)
        tot_sw += sw
        tot_dt += dt
    value = tot_sw / tot_dt
    sample = (f"per step one formulation (cycling 1..8), first {starts} starts, {sweeps} sweeps each, "
              f"FP64 oracle, OpenMP over starts")
    return {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * tot_dt / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": workload_config(args, w, world),
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------------------- distributed glue
_dist = None


def init_dist():
    global _dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        _dist = dist
    return rank, world, local


def barrier(world):
    if world > 1 and _dist is not None:
        _dist.barrier()


def _reduce(val, world, op):
    if world == 1 or _dist is None:
        return val
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else "cpu"
    t = torch.tensor([float(val)], dtype=torch.float64, device=dev)
    _dist.all_reduce(t, op=op)
    return t.item()


def reduce_max(val, world):
    return _reduce(val, world, _dist.ReduceOp.MAX if _dist else None)


def reduce_sum(val, world):
    return _reduce(val, world, _dist.ReduceOp.SUM if _dist else None)


# ---------------------------------------------------------------------------- shape scan
# The paper's GPU comparison (Section 5) on synthetic shapes: L1 variance with the L1 penalty
# (formulation 8), n = p / 200, p from 10^3 to 10^5, r in {1, 16, 256} starts; N(0,1) data, gamma
# by the Section 4.1 rule targeting 10 nonzeros, at most 100 sweeps, tol 1e-9.  Per shape: the
# GPU's sweeps*starts/s and single-solve latency, and the FP64 oracle's rate on the host cores on
# a bounded sample (its speedup is the ratio of the two).
SCAN_SHAPES = [(p, r) for p in (1000, 10000, 100000) for r in (1, 16, 256)]


def run_scan(args):
    import torch

    from oracle import oracle
    from paper_1212_4137_gb300 import build, inputs as I, spca
    build.build()
    oracle.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    kw = dict(s=10.0, gamma_target=True, calib=10, max_iter=100, tol=1e-9)
    for p, r in SCAN_SHAPES:
        n = p // 200
        A = I.gaussian_matrix(n, p, 900 + p).astype(np.float32)
        G = I.raw_starts(p, r, 901).astype(np.float32)
        Ad, Gd = torch.from_numpy(A).to(dev), torch.from_numpy(G).to(dev)
        h = spca.Handle(Ad, stream=stream.cuda_stream)
        for _ in range(args.warmup):
            h.solve(8, r, x0=Gd.data_ptr(), x0_device=True, **kw)
        lat, sweeps = [], 0
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            t1 = time.perf_counter()
            sweeps += h.solve(8, r, x0=Gd.data_ptr(), x0_device=True, **kw)["sweeps_total"]
            lat.append(1e3 * (time.perf_counter() - t1))
        dt = time.perf_counter() - t0
        h.close()
        # the oracle on a bounded sample: up to 16 starts, up to 20 sweeps
        ks, kk = min(r, 16), 20
        t1 = time.perf_counter()
        ref = oracle.solve(A.astype(np.float64), 8, G[:ks].astype(np.float64), s=10.0, gamma_target=True,
                           calib=10, max_iter=kk, tol=-1)
        odt = time.perf_counter() - t1
        gpu_rate, cpu_rate = sweeps / dt, int(ref.iters.sum()) / odt
        print(json.dumps({"scan": "L1-var L1-pen (formulation 8), n = p/200", "n": n, "p": p, "r": r,
                          "sweeps_starts_per_s": round(gpu_rate, 1), "solves_per_s": round(args.steps / dt, 2),
                          "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                                         "p99": round(float(np.percentile(lat, 99)), 3)},
                          "oracle_sweeps_starts_per_s": round(cpu_rate, 1), "oracle_cores": oracle.num_threads(),
                          "oracle_sample": f"{ks} starts x {kk} sweeps", "speedup": round(gpu_rate / cpu_rate, 1)}),
              flush=True)


# The economies-of-scale experiment of Section 4.2: the L0-penalised L2-variance formulation (5) on N(0,1)
# matrices with p = 1000, 2000, ..., 32000, l = 256 starting points, at most 10 sweeps each, run in
# batches of r = 1 (NAI), 4, 16, 64 and 256 (SFA) starts one batch after another.  The paper does not
# state n; here n = p / 10.  gamma by the Section 4.1 rule targeting 10 nonzeros over the first 5
# sweeps (the paper does not state gamma either); every start runs exactly 10 sweeps (tol < 0), so
# all batch sizes do the same work.  Per (p, r): sweeps*starts/s of the whole set of 256 starts and
# the speedup over r = 1; per p: the FP64 oracle's rate on one host core and on all of them, on a
# bounded sample.
ECON_PS = (1000, 2000, 4000, 8000, 16000, 32000)
ECON_RS = (1, 4, 16, 64, 256)


def run_scan_economies(args, l=256, sweeps=10):
    import torch

    from oracle import oracle
    from paper_1212_4137_gb300 import build, inputs as I, spca
    build.build()
    oracle.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    kw = dict(s=10.0, gamma_target=True, calib=5, max_iter=sweeps, tol=-1)
    for p in ECON_PS:
        n = p // 10
        A = I.gaussian_matrix(n, p, 4000 + p).astype(np.float32)
        G = I.raw_starts(p, l, 4001).astype(np.float32)
        Ad, Gd = torch.from_numpy(A).to(dev), torch.from_numpy(G).to(dev)
        h = spca.Handle(Ad, stream=stream.cuda_stream)
        rates = {}
        for r in ECON_RS:
            batches = [Gd[b:b + r] for b in range(0, l, r)]
            for _ in range(max(1, args.warmup)):
                h.solve(5, r, x0=batches[0].data_ptr(), x0_device=True, **kw)
            torch.cuda.synchronize(dev)
            best = None
            for _ in range(max(1, args.steps)):
                t0 = time.perf_counter()
                done = 0
                for xb in batches:
                    done += h.solve(5, r, x0=xb.data_ptr(), x0_device=True, **kw)["sweeps_total"]
                dt = time.perf_counter() - t0
                best = dt if best is None or dt < best else best
            assert done == l * sweeps
            rates[r] = l * sweeps / best
        h.close()
        # the oracle on a bounded sample: 4 starts on one core, 32 on all cores, 2 sweeps each
        A64 = A.astype(np.float64)
        okw = dict(s=10.0, gamma_target=True, calib=5, max_iter=2, tol=-1)
        t1 = time.perf_counter()
        o1 = oracle.solve(A64, 5, G[:4].astype(np.float64), nthreads=1, **okw)
        one = int(o1.iters.sum()) / (time.perf_counter() - t1)
        t1 = time.perf_counter()
        oa = oracle.solve(A64, 5, G[:32].astype(np.float64), **okw)
        allc = int(oa.iters.sum()) / (time.perf_counter() - t1)
        print(json.dumps({"scan": "economies of scale (Section 4.2), L0-pen L2-var (formulation 5)", "n": n, "p": p,
                          "l": l, "sweeps": sweeps,
                          "sweeps_starts_per_s": {f"BAT{r}": round(v, 1) for r, v in rates.items()},
                          "speedup_vs_NAI": {f"BAT{r}": round(v / rates[1], 2) for r, v in rates.items()},
                          "oracle_sweeps_starts_per_s": {"1 core": round(one, 1),
                                                         f"{oracle.num_threads()} cores": round(allc, 1)},
                          "oracle_sample": "4 starts (1 core) and 32 starts (all cores), 2 sweeps each"}),
              flush=True)


# The text corpora of Section 5 on a synthetic stand-in: a bag-of-words count matrix of the NYTimes
# corpus's shape (300,000 documents x 102,660 words, about 70 million stored counts; Zipf word
# popularity, log-normal document lengths, 5 planted topics), kept in compressed sparse rows.  The
# paper's settings: s = 5 (L0 forms; the L1 radius sqrt(5); the Section 4.1 rule targeting 5
# nonzeros for the penalty forms), 20 starts, at most 20 sweeps, tol 1e-6; and 256 starts for
# throughput.  Per (formulation, r): the GPU's sweeps*starts/s and single-solve latency, the share
# and DRAM-bound rate of v = A^T y, and (formulation 1) the FP64 oracle on a bounded sample.
TEXT = dict(n=300000, p=102660, nnz=70_000_000, seed=11, s=5, max_iter=20, tol=1e-6, calib=10)


def run_scan_text(args, forms=(1, 2, 3, 4, 5, 6, 7, 8), rs=(20, 256)):
    import torch

    from oracle import oracle
    from paper_1212_4137_gb300 import build, inputs as I, spca
    build.build()
    oracle.build()
    w = TEXT
    n, p = w["n"], w["p"]
    t0 = time.perf_counter()
    ip, ix, v = I.bag_of_words(n, p, w["nnz"], w["seed"])
    gen_s = time.perf_counter() - t0
    nnz = int(ip[-1])
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    h = spca.Handle((ip, ix, v, (n, p)), stream=stream.cuda_stream)
    create_s = time.perf_counter() - t0
    peaks = load_peaks()
    for r in rs:
        G = I.raw_starts(p, r, 12).astype(np.float32)
        Gd = torch.from_numpy(G).to(dev)
        for form in forms:
            kw = dict(s=float(w["s"]), max_iter=w["max_iter"], tol=w["tol"])
            if form >= 5:
                kw.update(gamma_target=True, calib=w["calib"])
            for _ in range(args.warmup):
                h.solve(form, r, x0=Gd.data_ptr(), x0_device=True, **kw)
            lat, sweeps = [], 0
            torch.cuda.synchronize(dev)
            ts = time.perf_counter()
            for _ in range(args.steps):
                t1 = time.perf_counter()
                sweeps += h.solve(form, r, x0=Gd.data_ptr(), x0_device=True, **kw)["sweeps_total"]
                lat.append(1e3 * (time.perf_counter() - t1))
            dt = time.perf_counter() - ts
            # one more solve with every kernel timed: shares, and v = A^T y against DRAM
            h.profile(True)
            out = h.solve(form, r, x0=Gd.data_ptr(), x0_device=True, **kw)
            kern = {name: h.profile_query(kid) for kid, name in spca.KERNEL_NAMES.items()}
            h.profile(False)
            tot = sum(ms for _, ms in kern.values()) or 1.0
            nv, msv = kern["v"]
            # algorithmic DRAM bytes of the sweeps' v = A^T y: A by columns once per sweep (index +
            # value, 8 B per stored entry), y of the active starts once, v written once; the gather
            # u = A x is queued once per sweep, so its launch count is the number of sweeps queued
            nsw = kern["u_sparse"][0]
            active = out["sweeps_total"]            # sweeps*starts = sum over sweeps of the active count
            vbytes = nsw * 8.0 * nnz + 4.0 * (n + p) * active
            line = {"scan": "text corpus (bag-of-words, NYTimes shape)", "form": form, "n": n, "p": p,
                    "nnz": nnz, "r": r, "s": w["s"], "max_iter": w["max_iter"], "tol": w["tol"],
                    "sweeps_starts_per_s": round(sweeps / dt, 1), "solves_per_s": round(args.steps / dt, 2),
                    "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                                   "p99": round(float(np.percentile(lat, 99)), 3)},
                    "sweeps_total": int(out["sweeps_total"]), "best_nnz": int(out["nnz"]),
                    "kernels_ms_share": {k: round(ms / tot, 4) for k, (_, ms) in kern.items()},
                    "v": {"sweeps": nsw, "launches": nv, "ms_per_sweep": round(msv / max(1, nsw), 4),
                          "achieved_gbs": round(vbytes / (msv / 1e3) / 1e9, 1) if msv > 0 else None,
                          "hbm_peak_gbs": peaks.get("hbm_gbs"),
                          "bytes": "8 B per stored entry per launch + 4 (n + p) B per active start"}}
            if form == 1 and r == rs[0]:
                A64 = sps_csr(ip, ix, v, n, p)
                t1 = time.perf_counter()
                ref = oracle.solve(A64, 1, G[:2].astype(np.float64), s=float(w["s"]), max_iter=2, tol=-1)
                odt = time.perf_counter() - t1
                line["oracle_sweeps_starts_per_s"] = round(int(ref.iters.sum()) / odt, 3)
                line["oracle_sample"] = "2 starts x 2 sweeps, FP64 CSR products, %d threads" % oracle.num_threads()
                line["generate_s"], line["create_s"] = round(gen_s, 2), round(create_s, 2)
            print(json.dumps(line), flush=True)
    # the first 5 sparse components (the paper's tables for the corpora): formulation 1, s = 5, 20
    # starts, each solve followed by the projection deflation of its x
    if 1 in forms and rs and rs[0] == 20:
        G = I.raw_starts(p, 20, 12).astype(np.float32)
        Gd = torch.from_numpy(G).to(dev)
        comps, t_comp = [], []
        for comp in range(5):
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            out = h.solve(1, 20, x0=Gd.data_ptr(), x0_device=True, s=float(w["s"]), max_iter=w["max_iter"],
                          tol=w["tol"])
            h.deflate(out["x"])
            torch.cuda.synchronize(dev)
            t_comp.append(1e3 * (time.perf_counter() - t1))
            comps.append({"objective": round(out["objective"], 4), "support": [int(j) for j in out["support"]]})
        print(json.dumps({"scan": "text corpus: first 5 components (formulation 1, s = 5, 20 starts, deflation "
                                  "after each)", "ms_per_component": [round(t, 2) for t in t_comp],
                          "components": comps}), flush=True)
    h.close()


# Few starts on the spiked workload (n = 5000, p = 20000, FP32; formulations 1 and 2, the settings
# of the benchmark): the streaming GEMV path (AUTO for r <= 8) and, at r = 1, the tensor-core
# engine beside it.  Per line: sweeps*starts/s, solve latency, and v = A^T y per sweep with its
# DRAM rate (A^T read once: 4 n p bytes, + 4 (n + p) bytes per start).
def run_scan_small_r(args):
    import torch

    from paper_1212_4137_gb300 import build, inputs as I, spca
    build.build()
    w = WORKLOADS[DEFAULT_WORKLOAD]
    n, p = w["n"], w["p"]
    A = make_inputs(w)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    h = spca.Handle(torch.from_numpy(A).to(dev), stream=stream.cuda_stream)
    peaks = load_peaks()
    for r, eng in ((1, spca.SPCA_ENGINE_AUTO), (1, spca.SPCA_ENGINE_TC), (4, spca.SPCA_ENGINE_AUTO),
                   (8, spca.SPCA_ENGINE_AUTO)):
        G = I.raw_starts(p, r, w["start_seed"]).astype(np.float32)
        Gd = torch.from_numpy(G).to(dev)
        for form in (1, 2):
            kw = dict(max_iter=w["max_iter"], tol=w["tol"], x0=Gd.data_ptr(), x0_device=True, engine=eng,
                      **solve_kwargs(w, form))
            for _ in range(args.warmup):
                h.solve(form, r, **kw)
            lat, sweeps = [], 0
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for _ in range(args.steps):
                t1 = time.perf_counter()
                sweeps += h.solve(form, r, **kw)["sweeps_total"]
                lat.append(1e3 * (time.perf_counter() - t1))
            dt = time.perf_counter() - t0
            h.profile(True, kernels=(spca.SPCA_K_V,))
            out = h.solve(form, r, **kw)
            nv, msv = h.profile_query(spca.SPCA_K_V)
            h.profile(False)
            vbytes = nv * 4.0 * n * p + 4.0 * (n + p) * out["sweeps_total"]
            print(json.dumps({"scan": "few starts, spiked 5000 x 20000", "form": form, "r": r,
                              "engine": {0: "auto", 1: "simt", 2: "tc"}[eng],
                              "sweeps_starts_per_s": round(sweeps / dt, 1),
                              "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                                             "p99": round(float(np.percentile(lat, 99)), 3)},
                              "v": {"launches": nv, "ms_per_launch": round(msv / max(1, nv), 4),
                                    "dram_gbs": round(vbytes / (msv / 1e3) / 1e9, 1) if msv > 0 else None,
                                    "hbm_peak_gbs": peaks.get("hbm_gbs"),
                                    "bytes": "4 n p per launch (A^T once) + 4 (n + p) per start-sweep"}}),
                  flush=True)
    h.close()


# The precision configuration: the spiked model at n = 20000, p = 50000 (FP32 A, 4 GB), 4096 starts,
# L0-constrained L2 and L1 variance (formulations 1 and 2), s = 100, at most 60 sweeps, tol 1e-9:
# plain FP32 sweeps against 20 low-precision sweeps followed by FP32 sweeps to the stopping rule,
# the low-precision sweeps on A's leading FP16 plane (11 significant bits) or on its FP8 E4M3 copy
# (4 significant bits, the tensor cores' 8-bit kind).  Per formulation and mode: the solve's wall time
# (CUDA events), sweeps*starts/s, and the best objective (FP64-class finalise) with its relative
# difference from the plain FP32 solve's.
# The precision configuration: spiked 20000 x 50000 (5 spikes of 100 nonzeros), FP32 A, 4096 starts,
# formulations 1 and 2 with s = 100, at most 60 sweeps, tol 1e-9.  Plain FP32 sweeps against
# schedules with a window of low-precision sweeps (A's 16-bit leading plane: 11 significant bits
# with per-row power-of-two scales; or the E4M3 copy of an FP8 handle: 4 significant bits with
# per-row and per-column power-of-two scales), FP32 accumulation throughout:
#   F10+L40: 10 FP32 sweeps (they decide which stationary point a start reaches), 40
#            low-precision sweeps, FP32 sweeps to the end;
#   L20:     the low-precision sweeps first (20), then FP32 (scan only).
# Per mode: solve time (CUDA events on the stream), sweeps*starts/s, the best objective and its
# relative difference from plain FP32's (the metric's bar is a shortfall of at most 1e-3).
PRECISION_MODES = (("fp32", "f32", {}),
                   ("fp16-plane F10+L40", "f32", {"lowp_first": 10, "lowp_sweeps": 40}),
                   ("fp8 F10+L40", "fp8", {"lowp_first": 10, "lowp_sweeps": 40}))
PRECISION_SCAN_EXTRA = (("fp16-plane L20", "f32", {"lowp_sweeps": 20}),
                        ("fp8 L20", "fp8", {"lowp_sweeps": 20}))


def precision_measure(modes, steps=1, warmup=1):
    import torch

    from paper_1212_4137_gb300 import build, inputs as I, spca
    build.build()
    n, p, r, s = 20000, 50000, 4096, 100
    A = I.spiked_matrix(n, p, I.spiked_thetas(n, p), 100, 20000, dtype=np.float32)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    Ad = torch.from_numpy(A).to(dev)
    handles = {"f32": spca.Handle(Ad, stream=stream.cuda_stream),
               "fp8": spca.Handle(Ad, stream=stream.cuda_stream, storage=spca.SPCA_FP8_E4M3_COLSCALED)}
    del A, Ad
    rows = []
    for form in (1, 2):
        base = None
        for name, hk, extra in modes:
            hh = handles[hk]
            kw = dict(s=float(s), seed=20001, max_iter=60, tol=1e-9, **extra)
            for _ in range(warmup):
                hh.solve(form, r, **kw)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ms, sweeps, out = 0.0, 0, None
            for _ in range(max(1, steps)):
                torch.cuda.synchronize(dev)
                e0.record(stream)
                out = hh.solve(form, r, **kw)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms += e0.elapsed_time(e1)
                sweeps += out["sweeps_total"]
            ms /= max(1, steps)
            row = {"form": form, "mode": name, "solve_ms": round(ms, 2),
                   "sweeps_starts_per_s": round(sweeps / max(1, steps) / (ms / 1e3), 1),
                   "sweeps_per_start": round(out["sweeps_total"] / r, 2), "best_objective": out["objective"],
                   "best_nnz": int(out["nnz"])}
            if base is None:
                base = row
            else:
                row["speedup_vs_fp32"] = round(base["solve_ms"] / ms, 3)
                row["best_rel_vs_fp32"] = (out["objective"] - base["best_objective"]) / abs(base["best_objective"])
            rows.append(row)
    for hh in handles.values():
        hh.close()
    return rows


def run_scan_precision(args):
    for row in precision_measure(PRECISION_MODES + PRECISION_SCAN_EXTRA, steps=args.steps, warmup=args.warmup):
        row = dict(row)
        row["scan"] = "precision, spiked 20000 x 50000, 4096 starts, s = 100, <= 60 sweeps, tol 1e-9"
        print(json.dumps(row), flush=True)


def _log_uniform(rng, lo, hi):
    return int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))


# The batching configuration: 256 independent spiked problems (k = 3 spikes, theta = (40, 30, 20)
# sqrt(n / p), 20 nonzeros each), n log-uniform in [200, 4000], p log-uniform in [500, 20000], FP32;
# per problem a uniform formulation, s uniform in [5, 100] (at most p), r = 64 starts, at most 100
# sweeps, tol 1e-9.  Modes: every problem solved one after another on its own handle; the same
# problems in one grouped solve (every sweep phase one launch over all 256, the tile shape from the
# tuning table); and the previous design, whole solves overlapping from 8 worker threads.
def draw_problems(count, seed, n_range=(200, 4000), p_range=(500, 20000), s_range=(5, 100), r=64, threads=16):
    """The batching configuration's problems: (name, A, form, solve kwargs, r); the matrices are
    generated on host threads (the generator's array operations release the interpreter lock)."""
    from paper_1212_4137_gb300 import inputs as I
    rng = np.random.default_rng(seed)
    spec = []
    for q in range(count):
        n, p = _log_uniform(rng, *n_range), _log_uniform(rng, *p_range)
        form = int(rng.integers(1, 9))
        s = float(min(int(rng.integers(s_range[0], s_range[1] + 1)), p))
        kw = dict(s=s, seed=6000 + q, max_iter=100, tol=1e-9)
        if form >= 5:
            kw.update(gamma_target=True, calib=10)
        spec.append((f"m{q}", n, p, form, kw))
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        mats = list(ex.map(lambda t: I.spiked_matrix(t[1], t[2], I.spiked_thetas(t[1], t[2], (40.0, 30.0, 20.0)), 20,
                                                     5000 + int(t[0][1:]), dtype=np.float32), spec))
    return [(name, A, form, kw, r) for (name, _, _, form, kw), A in zip(spec, mats)]


def run_scan_many(args, count=256, workers=8):
    import torch

    from paper_1212_4137_gb300 import build, serve, spca, tuning
    build.build()
    t0 = time.perf_counter()
    probs = draw_problems(count, 4)
    gen_s = time.perf_counter() - t0
    handles = [spca.Handle(A) for _, A, _, _, _ in probs]
    sum_np = int(sum(A.size for _, A, _, _, _ in probs))
    head = {"scan": f"many problems ({count} spiked, k = 3, n in [200, 4000], p in [500, 20000], r = 64)",
            "sum_n_p": sum_np, "host_generation_s": round(gen_s, 1)}

    def report(mode, dt, outs, extra=None):
        line = dict(head, mode=mode, wall_s=round(dt, 3),
                    sweeps_starts_per_s=round(sum(o["sweeps_total"] for o in outs) / dt, 1),
                    solves_per_s=round(count / dt, 1))
        line.update(extra or {})
        print(json.dumps(line), flush=True)

    # one after another
    for h, (_, _, form, kw, r) in list(zip(handles, probs))[:8]:   # warm-up
        h.solve(form, r, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    solo = [h.solve(form, r, **kw) for h, (_, _, form, kw, r) in zip(handles, probs)]
    report("one after another", time.perf_counter() - t0, solo)
    # one grouped solve
    g = spca.Group()
    req = [(h, form, r, kw) for h, (_, _, form, kw, r) in zip(handles, probs)]
    shape = tuning.choose(64) or (64, 4)
    g.solve(req, tiles=shape)   # warm-up: captures the graphs
    best = None
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        grouped = g.solve(req, tiles=shape)
        dt = time.perf_counter() - t0
        best = dt if best is None or dt < best else best
    rel = [abs(a["objective"] - b["objective"]) / max(1.0, abs(b["objective"])) for a, b in zip(grouped, solo)]
    # signed: the grouped best objective above (a better stationary point) or below the solo one
    sgn = [(a["objective"] - b["objective"]) / max(1.0, abs(b["objective"])) for a, b in zip(grouped, solo)]
    report(f"one grouped solve (tiles {shape[0]} x {shape[1]} stages)", best, grouped,
           {"max_rel_objective_diff_vs_one_after_another": float(max(rel)),
            "largest_rel_gain": float(max(sgn)), "largest_rel_shortfall": float(-min(sgn)),
            "problems_within_1e-5": int(sum(x <= 1e-5 for x in rel))})
    g.close()
    for h in handles:
        h.close()
    # the request loop: concurrent group sessions (a worker's session takes its share of the queue;
    # the sessions' launches overlap on the device), and whole solves on clones from concurrent
    # workers (the previous design)
    for mode, label in (("group", f"{workers} group sessions overlapping (request loop)"),
                        ("solve", f"{workers} workers, whole solves overlapping (request loop)")):
        with serve.Server(workers=workers, budget_bytes=64 << 30, mode=mode) as s:
            for name, A, _, _, _ in probs:
                s.register(name, A)
            for name, _, form, kw, r in probs[:workers]:
                s.submit(name, form, r, **kw).result()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            outs = [f.result() for f in [s.submit(name, form, r, **kw) for name, _, form, kw, r in probs]]
            report(label, time.perf_counter() - t0, outs)


# The tuning of the grouped contraction's tile shape (tuning.py): for each bucket of start counts a
# problem mix drawn like the batching configuration (64 problems, r = 16, 64, 256), every shape the
# library builds timed on one grouped solve (best of 2 after a warm-up); writes the table beside
# tuning.py and prints it.
def run_tune(args, count=64):
    import torch

    from paper_1212_4137_gb300 import build, spca, tuning
    build.build()
    table = {"how": "bench.py --tune: per bucket, one grouped solve of 64 problems drawn like the batching "
                    "configuration (n log-uniform in [200, 4000], p in [500, 20000], k = 3 spikes, uniform "
                    "formulation and s in [5, 100]) with r starts each; wall-clock ms, best of 2 after a warm-up",
             "gpu": torch.cuda.get_device_name(0), "buckets": {}}
    for r in (16, 64, 256):
        probs = draw_problems(count, 40 + r, r=r)
        handles = [spca.Handle(A) for _, A, _, _, _ in probs]
        g = spca.Group()
        req = [(h, form, rr, kw) for h, (_, _, form, kw, rr) in zip(handles, probs)]
        res = tuning.tune(g, req)
        table["buckets"][tuning.bucket(r)] = dict(res, problems=count, r=r)
        print(json.dumps({"tune": tuning.bucket(r), **res}), flush=True)
        g.close()
        for h in handles:
            h.close()
    with open(tuning.TABLE, "w") as fh:
        json.dump(table, fh, indent=1)


def spiked_on_device(n, p, thetas, nnz, seed, dev):
    """The spiked model A = sum_k theta_k u_k v_k^T + N(0,1) noise, built in FP32 on the device:
    the spike components from the seeded host generator (inputs.spike_components), the noise from a
    seeded torch generator (the serving configuration's matrices, 15 G entries in all, would take
    minutes to draw on the host)."""
    import torch

    from paper_1212_4137_gb300 import inputs as I
    U, V = I.spike_components(n, p, len(thetas), nnz, seed)
    Ut = torch.from_numpy(U * np.asarray(thetas, np.float64)).to(dev)
    Vt = torch.from_numpy(V).to(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    A = torch.empty((n, p), dtype=torch.float32, device=dev)
    rows = max(1, (1 << 27) // p)
    for r0 in range(0, n, rows):
        r1 = min(n, r0 + rows)
        blk = torch.randn((r1 - r0, p), generator=g, dtype=torch.float32, device=dev)
        blk += (Ut[r0:r1] @ Vt.T).float()
        A[r0:r1] = blk
    return A


class _Kept:
    """A registered handle the scan reuses across request loops (their close() leaves it open)."""

    def __init__(self, h):
        self._h = h

    def __getattr__(self, name):
        return getattr(self._h, name)

    def close(self):
        pass


# The serving configuration: 32 resident spiked matrices (5 spikes, theta = (40, 30, 20, 15, 10)
# sqrt(n / p), 50 nonzeros each), n log-uniform in [1000, 50000], p log-uniform in [2000, 100000],
# one of them pinned at 50000 x 100000, held in 16 bits (SPCA_FP16_RESIDENT: the leading FP16
# planes of A and A^T, 4 bytes per entry; the largest matrix's copy of A is 10 GB).  Requests: a
# uniform matrix, formulation 1..8, s uniform in [10, 200] (at most p), r uniform in {1, 16, 256},
# at most 100 sweeps, tol 1e-9.  Admission: the requests' working memory capped at 150 GB.  The
# request loop in group mode (`workers` group sessions, each admitting the waiting requests between
# segments of 4 sweeps) and, beside it, whole solves on clones.  A closed loop (every request
# queued at once) gives the capacity; then Poisson arrivals at 0.8 x capacity give the latency
# (p50 / p99 from submission to result).  Both runs of every mode take the same 2000 requests.
def run_scan_serving(args, mats=32, open_requests=2000,
                     modes=(("solve", 8, 1), ("group", 2, 1), ("group", 4, 4)), cap_gb=150):
    import torch

    from paper_1212_4137_gb300 import build, inputs as I, serve, spca
    build.build()
    spca.load()
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(5)
    shapes = [(50000, 100000)] + [(_log_uniform(rng, 1000, 50000), _log_uniform(rng, 2000, 100000))
                                  for _ in range(mats - 1)]
    t0 = time.perf_counter()
    free0 = torch.cuda.mem_get_info(dev)[0]
    kept = []
    for q, (n, p) in enumerate(shapes):
        A = spiked_on_device(n, p, I.spiked_thetas(n, p), 50, 7000 + q, dev)
        torch.cuda.synchronize(dev)
        kept.append(_Kept(spca.Handle(A, storage=spca.SPCA_FP16_RESIDENT)))
        del A
        torch.cuda.empty_cache()
    torch.cuda.synchronize(dev)
    gen_s = time.perf_counter() - t0
    resident = free0 - torch.cuda.mem_get_info(dev)[0]
    budget = cap_gb << 30
    head0 = {"scan": "serving", "matrices": mats, "sum_n_p": int(sum(n * p for n, p in shapes)),
             "largest": list(shapes[0]), "storage": "SPCA_FP16_RESIDENT (leading FP16 planes of A and A^T)",
             "resident_gb": round(resident / 2**30, 1), "member_budget_gb": cap_gb,
             "device_generation_and_create_s": round(gen_s, 1)}
    # one request list for every mode and for both runs of a mode, so that the Poisson rate is
    # 0.8 x the capacity measured on the same mix
    rq = np.random.default_rng(55)

    def request(i):
        name = f"s{int(rq.integers(0, mats))}"
        form = int(rq.integers(1, 9))
        s = float(min(int(rq.integers(10, 201)), shapes[int(name[1:])][1]))
        r = int(rq.choice([1, 16, 256]))
        kw = dict(s=s, seed=8000 + i, max_iter=100, tol=1e-9)
        if form >= 5:
            kw.update(gamma_target=True, calib=10)
        return name, form, r, kw

    warm = [request(i) for i in range(32)]
    reqs = [request(10000 + i) for i in range(open_requests)]
    unit_gaps = np.random.default_rng(56).exponential(1.0, open_requests)   # scaled by 1 / rate
    # size classes: thresholds on serve.request_cost that split the requests' total cost evenly
    costs = np.sort([serve.request_cost(*shapes[int(nm[1:])], r) for nm, _, r, _ in reqs])
    cum = np.cumsum(costs) / costs.sum()

    def thresholds(k):
        return [float(costs[np.searchsorted(cum, j / k)]) for j in range(1, k)]

    solve_rate = None   # the whole-solve mode's Poisson rate, also offered to the other modes
    for mode, workers, nclass in sorted(modes, key=lambda m: m[0] != "solve"):
        head = dict(head0, workers=workers, mode="group sessions, 4 sweeps per segment" if mode == "group"
                      else "whole solves on clones")
        if nclass > 1:
            head["size_classes"] = f"{nclass} (equal shares of the requests' total cost, one group per worker)"
        with serve.Server(workers=workers, budget_bytes=budget, mode=mode, classes=thresholds(nclass) if nclass > 1
                          else None, handle_factory=lambda A, stream=0, **kw: A) as srv:
            for q, h in enumerate(kept):
                srv.register(f"s{q}", h)
            for f in [srv.submit(nm, fm, r, **kw) for nm, fm, r, kw in warm]:
                f.result()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            outs = [f.result() for f in [srv.submit(nm, fm, r, **kw) for nm, fm, r, kw in reqs]]
            dt = time.perf_counter() - t0
            capacity = len(reqs) / dt
            print(json.dumps(dict(head, run="closed loop (capacity)", requests=len(reqs),
                                  solves_per_s=round(capacity, 2),
                                  sweeps_starts_per_s=round(sum(o["sweeps_total"] for o in outs) / dt, 1))), flush=True)
            runs = [("Poisson arrivals at 0.8 x capacity (the same requests)", 0.8 * capacity)]
            if mode == "solve":
                solve_rate = 0.8 * capacity
            elif solve_rate is not None:
                runs.append(("Poisson arrivals at the whole-solve mode's rate (the same requests)", solve_rate))
            for label, rate in runs:
                futs = []
                t0 = time.perf_counter()
                t_next = t0
                for (nm, fm, r, kw), g in zip(reqs, unit_gaps):
                    t_next += g / rate
                    while time.perf_counter() < t_next:
                        time.sleep(min(0.001, max(0.0, t_next - time.perf_counter())))
                    futs.append(srv.submit(nm, fm, r, **kw))
                t_last = time.perf_counter()
                outs = [f.result() for f in futs]
                dt = time.perf_counter() - t0
                lat = np.array([o["latency_ms"] for o in outs])
                by_r = {int(r): {"p50": round(float(np.percentile([o["latency_ms"] for o, q in zip(outs, reqs) if q[2] == r], 50)), 2),
                                 "p99": round(float(np.percentile([o["latency_ms"] for o, q in zip(outs, reqs) if q[2] == r], 99)), 2)}
                        for r in (1, 16, 256) if any(q[2] == r for q in reqs)}
                print(json.dumps(dict(head, run=label, requests=len(reqs),
                                      offered_per_s=round(rate, 2), arrivals_s=round(t_last - t0, 2),
                                      solves_per_s=round(len(reqs) / dt, 2),
                                      sweeps_starts_per_s=round(sum(o["sweeps_total"] for o in outs) / dt, 1),
                                      latency_ms={"p50": round(float(np.percentile(lat, 50)), 2),
                                                  "p99": round(float(np.percentile(lat, 99)), 2)},
                                      latency_by_r_ms=by_r,
                                      queue_ms_p50=round(float(np.percentile([o["queue_ms"] for o in outs], 50)), 2))),
                      flush=True)
    for h in kept:
        h._h.close()


def sps_csr(ip, ix, v, n, p):
    import scipy.sparse as sps
    return sps.csr_matrix((v.astype(np.float64), ix, ip), shape=(n, p))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=tuple(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # for profiler captures: a subset of the formulations, no end-to-end pass
    ap.add_argument("--forms", type=str, default=None, help="comma-separated formulations (default: all 8)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the precision configuration's extra key")
    # the paper's shape scan (one JSON line per shape) instead of the benchmark line
    ap.add_argument("--scan", choices=("paper-shapes", "text-corpus", "few-starts", "precision", "many-problems",
                                       "serving", "economies"), default=None)
    ap.add_argument("--rs", type=str, default=None, help="text-corpus scan: comma-separated start counts")
    ap.add_argument("--tune", action="store_true", help="measure the grouped contraction's tile shapes")
    args = ap.parse_args()
    if args.tune:
        run_tune(args)
        return
    if args.scan == "text-corpus":
        kw = {}
        if args.forms:
            kw["forms"] = tuple(int(t) for t in args.forms.split(","))
        if args.rs:
            kw["rs"] = tuple(int(t) for t in args.rs.split(","))
        run_scan_text(args, **kw)
        return
    if args.scan == "few-starts":
        run_scan_small_r(args)
        return
    if args.scan == "precision":
        run_scan_precision(args)
        return
    if args.scan == "many-problems":
        run_scan_many(args)
        return
    if args.scan == "serving":
        run_scan_serving(args)
        return
    if args.scan == "economies":
        run_scan_economies(args)
        return
    if args.scan:
        run_scan(args)
        return
    rank, world, local = init_dist()
    w = dict(WORKLOADS[args.workload])
    if args.forms:
        w["forms"] = tuple(int(t) for t in args.forms.split(","))
    if args.impl == "reference":
        line = run_reference(args, w, rank, world)
    else:
        line = run_ours(args, w, rank, world, local)
        if line is not None and world == 1 and not args.no_cpu_baseline:
            from paper_1212_4137_gb300 import inputs as I
            G = I.raw_starts(w["p"], w["r"], w["start_seed"]).astype(np.float32)
            line["cpu_baseline"] = cpu_baseline(w, make_inputs(w), G)
        if line is not None and world == 1 and not args.no_precision and args.workload == DEFAULT_WORKLOAD:
            # the precision configuration (not part of the timed region above): one solve per mode
            # and formulation after one warm-up
            line["precision"] = {
                "workload": "spiked 20000 x 50000, 4096 starts, formulations 1 and 2, s = 100, <= 60 sweeps, "
                            "tol 1e-9; low-precision window of 40 sweeps after 10 FP32 sweeps",
                "results": precision_measure(PRECISION_MODES)}
    if line is not None:
        print(json.dumps(line), flush=True)
    if _dist is not None:
        _dist.destroy_process_group()


if __name__ == "__main__":
    main()
