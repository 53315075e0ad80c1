#!/usr/bin/env python
"""Benchmark of the HMatrix-matrix evaluation Y = K~ W on GB300 (one JSON line on stdout).

Default workload: H2 geometric admissibility, N = 65536 points in d = 8 from a
10-component Gaussian mixture, Gaussian kernel h = 1, leaf size 128, ID tolerance
1e-5, rank <= 128, W = 65536 x 256 N(0, 1), FP64 evaluation. The HMatrix is built
by the library's inspector (hmat_build); a step is one full evaluation (near
field, upward pass, coupling, downward pass) through hmat_eval.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun every rank evaluates its own copy of the HMatrix on its own GPU
(independent problems, no collective on the data path): value = columns of all
ranks / the slowest rank's time ("weak" scaling). --impl reference times the FP64
CPU oracle on the host cores on a bounded column sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "H-matmul cols/s and % HBM roofline, mixed vs FP64 at 1e-6 err; p50/p99 latency"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", default="h2_gmm8d_n65536")
    ap.add_argument("--n", type=int, default=None, help="reduced point count (small profiling cases)")
    ap.add_argument("--q", type=int, default=None, help="override the number of right-hand-side columns")
    ap.add_argument("--cpu-baseline", choices=["auto", "off"], default="auto")
    ap.add_argument("--mixed", choices=["on", "off"], default="on",
                    help="also time the mixed-precision tensor-core mode on the same HMatrix")
    ap.add_argument("--batch", choices=["on", "off"], default="on",
                    help="also time the batched mode: 64 HMatrices of uneven N, d, kernel, leaf size and q")
    ap.add_argument("--serve", choices=["short", "full", "off"], default="full",
                    help="also run the serving mode: a Poisson request stream on resident HMatrices "
                         "(short: 4 matrices N = 16K..128K, 6 s; full: 8 matrices N = 16K..1M, 2000 req/s, 60 s)")
    ap.add_argument("--precision", choices=["on", "off"], default="on",
                    help="time the precision-mode recipe (N=262144 inverse multiquadric, q=512), FP64 vs mixed")
    ap.add_argument("--otf", choices=["on", "off"], default="on",
                    help="near blocks evaluated on the fly (FP64) on the headline recipe")
    ap.add_argument("--matvec", choices=["on", "off"], default="on",
                    help="time the matrix-vector recipe (N=262144, kernel 1/r, q=1), FP64 vs mixed")
    ap.add_argument("--hss", choices=["on", "off"], default="on",
                    help="time the latency-bound HSS recipe (N=2048, q=16, FP64): microseconds per evaluation")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target length of the CPU baseline sample")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed helpers

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def aggregate(dist: "Dist", columns_per_rank: int, ms_local: float) -> tuple:
    """Whole-job throughput: the columns all ranks processed over the slowest rank's time per step.
    Every rank evaluates its own replica of the problem (no collective on the data path)."""
    ms = dist.max(ms_local)
    return dist.world * columns_per_rank / (ms / 1e3), ms


# ----------------------------------------------------------------------------- clocks during the timed region

CLOCK_FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                "clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, device_index: int):
        self.path = tempfile.mktemp(prefix="hmat_clocks_", suffix=".csv")
        self.proc = None
        self.device_index = device_index

    def start(self):
        try:
            ident = self._gpu_id()
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={ident}", f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def _gpu_id(self) -> str:
        import torch
        try:
            u = str(torch.cuda.get_device_properties(self.device_index).uuid)
            return u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            return vis.split(",")[self.device_index] if vis else str(self.device_index)

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[4:8]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm

def workload(args):
    from workloads import WORKLOADS, reduced
    w = WORKLOADS[args.workload]
    if args.n is not None or args.q is not None:
        w = reduced(w, args.n or w.n, q=args.q)
    return w


def build_params(w):
    return dict(kernel=w.kernel, kernel_param=w.kernel_param, admissibility=w.admissibility,
                leaf_size=w.leaf_size, tol=w.tol, max_rank=w.max_rank, eta=w.eta, sample_seed=w.sample_seed)


def run_gpu(args, dist: Dist) -> None:
    import numpy as np
    import torch

    from paper_1812_07152_gb300 import build as hbuild
    hbuild.build()
    import paper_1812_07152_gb300 as hp
    from workloads import make_points, normal_rhs

    torch.cuda.set_device(dist.local_rank)
    dist.init("nccl")
    w = workload(args)
    X = make_points(w)
    t0 = time.perf_counter()
    flags = hp.HMAT_LOAD_MIXED if args.mixed == "on" else 0
    dev = hp.DeviceHMatrix.build(X, flags=flags, **build_params(w))
    t_build = time.perf_counter() - t0
    info = dev.info
    q = w.q
    W_host = torch.from_numpy(normal_rhs(w.n, q, w.rhs_seed)).pin_memory()
    W = W_host.cuda()
    Y = torch.empty_like(W)
    dev.reserve(q)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    tune = hp.hmat_autotune(dev.handle, q, hp.HMAT_MODE_FP64, stream)
    tune["seconds"] = round(time.perf_counter() - t0, 2)

    for _ in range(args.warmup):
        hp.hmat_eval(dev.handle, W, Y, q, hp.HMAT_MODE_FP64, stream)
    torch.cuda.synchronize()
    if dev.poll() != hp.HMAT_OK:
        raise RuntimeError("device status error during warm-up")

    clocks = ClockSampler(dist.local_rank)
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    hp.hmat_profile(dev.handle, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        hp.hmat_eval(dev.handle, W, Y, q, hp.HMAT_MODE_FP64, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    ms_local = e0.elapsed_time(e1) / args.steps
    phases = hp.hmat_phase_times(dev.handle)
    hp.hmat_profile(dev.handle, False)
    value, ms = aggregate(dist, q, ms_local)
    if dev.poll() != hp.HMAT_OK:
        raise RuntimeError("device status error during the timed steps")

    mixed = run_mixed(args, dev, W, Y, q, info, stream, dist) if args.mixed == "on" else None

    # end to end: host W -> device, evaluate, device Y -> host, every step (pinned host buffers)
    Y_host = torch.empty_like(W_host).pin_memory()
    e2e = {}
    modes = [("fp64", hp.HMAT_MODE_FP64)] + ([("mixed", hp.HMAT_MODE_MIXED)] if mixed is not None else [])
    for name, mode in modes:
        hp.hmat_eval_host(dev.handle, W_host, Y_host, mode, stream)
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hp.hmat_eval_host(dev.handle, W_host, Y_host, mode, stream)
        e2e[name] = dist.world * q / dist.max((time.perf_counter() - t0) / args.steps)
    if mixed is not None:
        mixed["e2e"] = {"value": round(e2e["mixed"], 3), "unit": "cols/s", "h2d_bytes_per_step": int(W_host.numel() * 8),
                        "d2h_bytes_per_step": int(Y_host.numel() * 8)}

    e2e_value = e2e["fp64"]

    # roofline of the dominant kernel: the FP64 near-field grouped GEMM (bound by the DFMA pipe)
    # (a phase may be split into one launch per row-tile size: the unit is one evaluation's near field)
    near_ms, near_launches = phases["near"]
    near_ms_per_eval = near_ms / args.steps
    near_flops = 2.0 * q * info["near_values"]
    peak_gflops = hp.hmat_measure_fp64_peak()
    achieved_tflops = near_flops / (near_ms_per_eval / 1e3) / 1e12
    total_flops = 2.0 * q * (info["near_values"] + 2 * info["basis_values"] + info["coupling_values"])
    bytes_step = 8.0 * (info["near_values"] + info["basis_values"] + info["coupling_values"]) + 2 * 8.0 * w.n * q
    launches = sum(c for _, c in phases.values())

    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "cols/s",
        "n_gpus": dist.world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {
            "workload": w.name, "n": w.n, "d": w.d, "points": "10-component Gaussian mixture" if w.points == "gmm"
            else "uniform", "q": q, "kernel": f"{w.kernel} {w.kernel_param}", "admissibility": w.admissibility,
            "leaf_size": w.leaf_size, "tol": w.tol, "max_rank": w.max_rank, "mode": "fp64",
            "near_entries": info["near_entries"], "far_entries": info["far_entries"],
            "near_values": info["near_values"], "basis_values": info["basis_values"],
            "coupling_values": info["coupling_values"], "sum_rank": info["sum_rank"],
            "inspector_s": round(t_build, 2), "l2": "inputs larger than L2 (near blocks "
            f"{8 * info['near_values'] / 1e9:.1f} GB read every step)",
            "parallelism": f"replicas x{dist.world}",
        },
        "gflops": round(total_flops / (ms / 1e3) / 1e9, 2),
        "phases_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in phases.items() if v[1] > 0},
        "roofline": {
            "bound": "alu", "kernel": "k_grouped_gemm<double> (near field, tuned column tile)",
            "launches_per_eval": near_launches // args.steps,
            "achieved": round(achieved_tflops, 4), "peak": round(peak_gflops / 1e3, 4), "unit": "TFLOP/s",
            "frac": round(achieved_tflops / (peak_gflops / 1e3), 4),
            "traffic": measured_traffic("fp64_near", info["near_values"]),
            "peak_source": "FP64 DFMA loop measured in this run (hmat_measure_fp64_peak); nominal 1.25",
            "step_bytes": bytes_step,
            "step_hbm_bound_ms": round(bytes_step / (measured_peaks()["hbm_gbs"] * 1e9) * 1e3, 3),
        },
        "e2e": {"value": round(e2e_value, 3), "unit": "cols/s", "h2d_bytes_per_step": int(W_host.numel() * 8),
                "d2h_bytes_per_step": int(Y_host.numel() * 8)},
        "gpu_launches": launches,
        "clocks": clk,
        "autotune": {"fp64": tune},
    }
    if mixed is not None:
        line["autotune"]["mixed"] = mixed.pop("autotune")
        line["mixed"] = mixed
    dev.close()

    line["inspector_reuse"] = run_inspector_reuse(w, X)
    if args.otf == "on":
        line["near_on_the_fly"] = run_near_otf(w, X, dist, ms, info)
    if args.precision == "on":
        line["precision"] = run_precision(args, dist, peak_gflops)
    if args.matvec == "on":
        line["matvec"] = run_matvec(args, dist, peak_gflops)

    if args.hss == "on":
        line["hss"] = run_hss(args, dist)
    if args.batch == "on":
        line["batch"] = run_batch(args, dist)
    if args.serve != "off":
        line["serving"] = run_serving(args, dist)
    if dist.rank == 0 and dist.world == 1 and args.cpu_baseline == "auto":
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    dist.close()


def run_mixed(args, dev, W, Y64, q, info, stream, dist) -> dict:
    """Times the mixed-precision mode (tensor-core near field) on the same HMatrix and W;
    its error is measured against this run's FP64 result."""
    import torch
    import paper_1812_07152_gb300 as hp
    Ym = torch.empty_like(W)
    t0 = time.perf_counter()
    tune = hp.hmat_autotune(dev.handle, q, hp.HMAT_MODE_MIXED, stream)
    tune["seconds"] = round(time.perf_counter() - t0, 2)
    for _ in range(args.warmup):
        hp.hmat_eval(dev.handle, W, Ym, q, hp.HMAT_MODE_MIXED, stream)
    torch.cuda.synchronize()
    dist.barrier()
    hp.hmat_profile(dev.handle, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        hp.hmat_eval(dev.handle, W, Ym, q, hp.HMAT_MODE_MIXED, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    ms = dist.max(e0.elapsed_time(e1) / args.steps)
    phases = hp.hmat_phase_times(dev.handle)
    hp.hmat_profile(dev.handle, False)
    if dev.poll() != hp.HMAT_OK:
        raise RuntimeError("device status error during the mixed-precision steps")
    err = float(torch.linalg.norm(Ym - Y64) / torch.linalg.norm(Y64))
    serial = serial_phases(dev.handle, W, Ym, q, hp.HMAT_MODE_MIXED, stream, args.steps)
    roof = tc_near_roofline(info, q, serial["near"])
    roof["near_ms_beside_far_chain"] = round(phases["near"][0] / args.steps, 4)
    return {"value": round(dist.world * q / (ms / 1e3), 3), "unit": "cols/s", "ms_per_step": round(ms, 4),
            "error_vs_fp64": err, "dtype": "f16 hi+lo split, f32 accumulate",
            "phases_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in phases.items() if v[1] > 0},
            "phases_serialised_ms_per_step": serial,
            "launches_per_eval": sum(c for _, c in phases.values()) // args.steps,
            "gpu_launches": sum(c for _, c in phases.values()), "roofline": roof, "autotune": tune}


def serial_phases(dev_handle, W, Y, q, mode, stream, steps: int) -> dict:
    """Per-launch device times with the mixed mode's far chain serialised on the caller's stream (hmat_profile
    mode 2), so that each launch is timed alone: {phase: ms per evaluation}."""
    import torch
    import paper_1812_07152_gb300 as hp
    hp.hmat_profile(dev_handle, 2)
    for _ in range(steps):
        hp.hmat_eval(dev_handle, W, Y, q, mode, stream)
    torch.cuda.synchronize()
    ph = hp.hmat_phase_times(dev_handle)
    hp.hmat_profile(dev_handle, False)
    return {k: round(v[0] / steps, 4) for k, v in ph.items() if v[1] > 0}


def tc_near_roofline(info, q: int, near_ms: float) -> dict:
    """Roofline of the tensor-core near field (k_tc<0>) over one evaluation: executed flops (three FP16
    products per stored value), useful flops (one product, what the FP64 form computes) and the algorithmic
    bytes (D hi/lo once, the W split once, Y written once in FP64), each against its measured peak."""
    nv = info["near_values"]
    n = w_rows(info)
    exec_flops = 3 * 2.0 * q * nv
    useful_flops = 2.0 * q * nv
    alg_bytes = 4.0 * nv + 4.0 * n * q + 8.0 * n * q
    peaks = measured_peaks()
    t_tensor = exec_flops / (peaks["bf16_tflops"] * 1e12) * 1e3
    t_hbm = alg_bytes / (peaks["hbm_gbs"] * 1e9) * 1e3
    sec = near_ms / 1e3
    tensor_achieved = exec_flops / sec / 1e12
    hbm_achieved = alg_bytes / sec / 1e9
    if t_tensor >= t_hbm:
        roof = {"bound": "tensor", "achieved": round(tensor_achieved, 2), "peak": peaks["bf16_tflops"],
                "unit": "TFLOP/s"}
    else:
        roof = {"bound": "hbm", "achieved": round(hbm_achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    roof.update({"frac": round(roof["achieved"] / roof["peak"], 4),
                 "tensor_frac_executed": round(tensor_achieved / peaks["bf16_tflops"], 4),
                 "tensor_frac_useful": round(useful_flops / sec / 1e12 / peaks["bf16_tflops"], 4),
                 "hbm_frac": round(hbm_achieved / peaks["hbm_gbs"], 4),
                 "near_ms_per_eval": round(near_ms, 4), "traffic": measured_traffic("mixed_near", nv),
                 "algorithmic_bytes": alg_bytes, "executed_flops": exec_flops,
                 "kernel": "k_tc<0> (tcgen05 near field)", "peak_source": peaks["source"] + " (MEASURED_PEAKS.json)",
                 "t_tensor_ms": round(t_tensor, 4), "t_hbm_ms": round(t_hbm, 4)})
    return roof


def run_inspector_reuse(w, X) -> dict:
    """Inspector reuse (Section 3.2): the plan (tree + near/far lists) is built once, then the
    HMatrix is recompressed for the recipe's tolerance and for a ten times looser one without
    rebuilding it; times in seconds, each recompression including its load to the GPU."""
    import paper_1812_07152_gb300 as hp
    t0 = time.perf_counter()
    plan = hp.hmat_plan_create(X, admissibility=w.admissibility, leaf_size=w.leaf_size, eta=w.eta)
    t_plan = time.perf_counter() - t0
    out = {"plan_s": round(t_plan, 3), "recompress_s": {}, "recompress_gpu_id_s": {}}
    try:
        for tol in (w.tol, 10 * w.tol):
            for key, flags in (("recompress_s", 0), ("recompress_gpu_id_s", hp.HMAT_BUILD_ID_GPU)):
                t0 = time.perf_counter()
                h = hp.hmat_plan_build(plan, w.kernel, w.kernel_param, tol, w.max_rank, sample_seed=w.sample_seed,
                                       flags=flags)
                out[key][f"{tol:g}"] = round(time.perf_counter() - t0, 3)
                out.setdefault("sum_rank", {})[f"{tol:g} {key}"] = hp.hmat_info(h)["sum_rank"]
                hp.hmat_free(h)
    finally:
        hp.hmat_plan_free(plan)
    return out


def run_near_otf(w, X, dist, stored_ms, stored_info) -> dict:
    """Near blocks evaluated on the fly (HMAT_BUILD_NEAR_OTF) on the headline recipe, FP64 mode: the
    handle holds the points instead of the near blocks; time per evaluation (autotuned, 2 steps after
    a warm-up) against the stored form, and the device bytes each holds."""
    import torch
    import paper_1812_07152_gb300 as hp
    from workloads import normal_rhs
    q = w.q
    t0 = time.perf_counter()
    h = hp.hmat_build(X, flags=hp.HMAT_BUILD_NEAR_OTF, **build_params(w))
    t_build = time.perf_counter() - t0
    try:
        info = hp.hmat_info(h)
        stream = torch.cuda.current_stream()
        W = torch.from_numpy(normal_rhs(w.n, q, w.rhs_seed)).cuda()
        Y = torch.empty_like(W)
        tune = hp.hmat_autotune(h, q, hp.HMAT_MODE_FP64, stream)
        hp.hmat_eval(h, W, Y, q, hp.HMAT_MODE_FP64, stream)
        torch.cuda.synchronize()
        dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        steps = 2
        e0.record(stream)
        for _ in range(steps):
            hp.hmat_eval(h, W, Y, q, hp.HMAT_MODE_FP64, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = dist.max(e0.elapsed_time(e1) / steps)
        if hp.hmat_status_poll(h) != hp.HMAT_OK:
            raise RuntimeError("device status error in the on-the-fly steps")
        return {"mode": "fp64", "value": round(dist.world * q / (ms / 1e3), 3), "unit": "cols/s",
                "ms_per_step": round(ms, 3), "steps": steps, "stored_ms_per_step": round(stored_ms, 3),
                "device_bytes": info["device_bytes"], "near_block_bytes_not_held": 8 * info["near_values"],
                "stored_handle_device_bytes_incl_mixed_copy": stored_info["device_bytes"],
                "build_s": round(t_build, 2), "autotune": tune}
    finally:
        hp.hmat_free(h)


def run_precision(args, dist, fp64_peak: float) -> dict:
    """Precision mode on its own recipe: N = 262144 uniform points in [0,1]^3, inverse multiquadric
    1/sqrt(r^2 + 0.01), geometric admissibility, leaf 256, ID tol 1e-7, q = 512. The mixed form (FP16 hi+lo
    tensor-core near field, FP32 far field, FP64 output sums) against the FP64 form on the same GPU; its error
    is measured against this run's FP64 result."""
    import torch
    import paper_1812_07152_gb300 as hp
    from workloads import WORKLOADS, make_points, normal_rhs
    w = WORKLOADS["h2_imq3d_n262144"]
    t0 = time.perf_counter()
    dev = hp.DeviceHMatrix.build(make_points(w), flags=hp.HMAT_LOAD_MIXED, **build_params(w))
    t_build = time.perf_counter() - t0
    info = dev.info
    q = w.q
    W = torch.from_numpy(normal_rhs(w.n, q, w.rhs_seed)).cuda()
    Y64 = torch.empty_like(W)
    Ym = torch.empty_like(W)
    stream = torch.cuda.current_stream()
    dev.reserve(q)
    out = {"workload": w.name, "n": w.n, "q": q, "kernel": f"{w.kernel} {w.kernel_param}", "leaf_size": w.leaf_size,
           "tol": w.tol, "max_rank": w.max_rank, "near_values": info["near_values"], "sum_rank": info["sum_rank"],
           "inspector_s": round(t_build, 2), "unit": "cols/s"}
    tunes = {}
    # both forms are timed over --steps evaluations (an FP64 evaluation takes about 1.6 s)
    for name, mode, Y in (("fp64", hp.HMAT_MODE_FP64, Y64), ("mixed", hp.HMAT_MODE_MIXED, Ym)):
        steps = args.steps
        tunes[name] = hp.hmat_autotune(dev.handle, q, mode, stream)
        for _ in range(1 if mode == hp.HMAT_MODE_FP64 else args.warmup):
            hp.hmat_eval(dev.handle, W, Y, q, mode, stream)
        torch.cuda.synchronize()
        dist.barrier()
        hp.hmat_profile(dev.handle, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            hp.hmat_eval(dev.handle, W, Y, q, mode, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = dist.max(e0.elapsed_time(e1) / steps)
        phases = hp.hmat_phase_times(dev.handle)
        hp.hmat_profile(dev.handle, False)
        if dev.poll() != hp.HMAT_OK:
            raise RuntimeError(f"device status error in the precision-mode {name} steps")
        near_ms = phases["near"][0] / steps
        out[name] = {"value": round(dist.world * q / (ms / 1e3), 2), "ms_per_step": round(ms, 4), "steps": steps,
                     "phases_ms_per_step": {k: round(v[0] / steps, 4) for k, v in phases.items() if v[1] > 0},
                     "launches_per_eval": sum(c for _, c in phases.values()) // steps}
        if mode == hp.HMAT_MODE_FP64:
            achieved = 2.0 * q * info["near_values"] / (near_ms / 1e3) / 1e12
            out[name]["roofline"] = {"bound": "alu", "achieved": round(achieved, 4), "unit": "TFLOP/s",
                                     "peak": round(fp64_peak / 1e3, 4), "frac": round(achieved / (fp64_peak / 1e3), 4),
                                     "kernel": "k_grouped_gemm<double> (near field)"}
        else:
            serial = serial_phases(dev.handle, W, Y, q, mode, stream, steps)
            out[name]["phases_serialised_ms_per_step"] = serial
            out[name]["roofline"] = tc_near_roofline(info, q, serial["near"])
            out[name]["roofline"]["near_ms_beside_far_chain"] = round(near_ms, 4)
    out["mixed"]["error_vs_fp64"] = float(torch.linalg.norm(Ym - Y64) / torch.linalg.norm(Y64))
    out["mixed_over_fp64"] = round(out["mixed"]["value"] / out["fp64"]["value"], 2)
    out["autotune"] = tunes
    dev.close()
    # the same compression with the row IDs on the GPU (one CTA per node of a level)
    t0 = time.perf_counter()
    h = hp.hmat_build(make_points(w), flags=hp.HMAT_BUILD_ID_GPU, **build_params(w))
    out["inspector_gpu_id_s"] = round(time.perf_counter() - t0, 2)
    out["sum_rank_gpu_id"] = hp.hmat_info(h)["sum_rank"]
    hp.hmat_free(h)
    return out


def run_matvec(args, dist, peak_gflops: float) -> dict:
    """Matrix-vector form of the comparison with SMASH (Section 4.1): N = 262144 uniform points in [0,1]^3,
    kernel 1/r (0 for coincident points), geometric admissibility, leaf 256, ID tol 1e-6, q = 1. The FP64 near
    field is bound by the FP64 pipe even at q = 1 (q/4 flop per stored byte against a ridge of 0.18); the mixed
    near field reads 4 B per stored value and is bound by HBM."""
    import torch
    import paper_1812_07152_gb300 as hp
    from workloads import WORKLOADS, make_points, normal_rhs
    w = WORKLOADS["h2_invdist3d_n262144"]
    t0 = time.perf_counter()
    dev = hp.DeviceHMatrix.build(make_points(w), flags=hp.HMAT_LOAD_MIXED, **build_params(w))
    t_build = time.perf_counter() - t0
    info = dev.info
    q = w.q
    W = torch.from_numpy(normal_rhs(w.n, q, w.rhs_seed)).cuda()
    Ys = {"fp64": torch.empty_like(W), "mixed": torch.empty_like(W)}
    stream = torch.cuda.current_stream()
    dev.reserve(q)
    nv = info["near_values"]
    peaks = measured_peaks()
    out = {"workload": w.name, "n": w.n, "q": q, "kernel": "1/r", "leaf_size": w.leaf_size, "tol": w.tol,
           "near_values": nv, "coupling_values": info["coupling_values"], "sum_rank": info["sum_rank"],
           "coupling_engine": info["coupling_engine"], "inspector_s": round(t_build, 2), "unit": "cols/s"}
    steps = max(args.steps, 20)
    for name, mode in (("fp64", hp.HMAT_MODE_FP64), ("mixed", hp.HMAT_MODE_MIXED)):
        hp.hmat_autotune(dev.handle, q, mode, stream)
        for _ in range(args.warmup):
            hp.hmat_eval(dev.handle, W, Ys[name], q, mode, stream)
        torch.cuda.synchronize()
        dist.barrier()
        hp.hmat_profile(dev.handle, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            hp.hmat_eval(dev.handle, W, Ys[name], q, mode, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = dist.max(e0.elapsed_time(e1) / steps)
        phases = hp.hmat_phase_times(dev.handle)
        hp.hmat_profile(dev.handle, False)
        if dev.poll() != hp.HMAT_OK:
            raise RuntimeError(f"device status error in the matrix-vector {name} steps")
        near_ms = phases["near"][0] / steps
        if mode == hp.HMAT_MODE_FP64:
            achieved = 2.0 * q * nv / (near_ms / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak_gflops / 1e3, 4),
                    "unit": "TFLOP/s", "frac": round(achieved / (peak_gflops / 1e3), 4),
                    "kernel": "k_grouped_gemm<double> 1-column tiles (near field)"}
        else:
            serial = serial_phases(dev.handle, W, Ys[name], q, mode, stream, steps)
            near_ms = serial["near"]
            alg = 4.0 * nv + 8.0 * w.n * q * 2
            achieved = alg / (near_ms / 1e3) / 1e9
            roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": round(achieved / peaks["hbm_gbs"], 4), "algorithmic_bytes": alg,
                    "kernel": "k_tc (tcgen05 near field, 16-column tile)", "peak_source": peaks["source"]}
        out[name] = {"value": round(dist.world * q / (ms / 1e3), 1), "ms_per_step": round(ms, 4), "steps": steps,
                     "phases_ms_per_step": {k: round(v[0] / steps, 4) for k, v in phases.items() if v[1] > 0},
                     "launches_per_eval": sum(c for _, c in phases.values()) // steps, "roofline": roof}
        if mode == hp.HMAT_MODE_MIXED:
            out[name]["phases_serialised_ms_per_step"] = serial
    out["mixed"]["error_vs_fp64"] = float(torch.linalg.norm(Ys["mixed"] - Ys["fp64"]) / torch.linalg.norm(Ys["fp64"]))
    dev.close()
    return out


def run_hss(args, dist) -> dict:
    """Latency of the small HSS recipe: N = 2048 uniform points in [0,1]^3, weak admissibility (every pair of
    siblings far), Gaussian h = 0.5, leaf 64, ID tol 1e-6, rank <= 64, q = 16, FP64. Its work is a few MFLOP, so
    the time is launch latency: microseconds per evaluation through hmat_eval, and replayed as a one-member
    batch (one CUDA graph launch per evaluation)."""
    import torch
    import paper_1812_07152_gb300 as hp
    from workloads import WORKLOADS, make_points, normal_rhs
    w = WORKLOADS["hss_uniform3d_n2048"]
    h = hp.hmat_build(make_points(w), **build_params(w))
    try:
        info = hp.hmat_info(h)
        q = w.q
        W = torch.from_numpy(normal_rhs(w.n, q, w.rhs_seed)).cuda()
        Y = torch.empty_like(W)
        stream = torch.cuda.current_stream()
        hp.hmat_reserve(h, q)
        steps = max(200, 10 * args.steps)

        def timed(fn):
            for _ in range(max(args.warmup, 10)):
                fn()
            torch.cuda.synchronize()
            dist.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return dist.max(e0.elapsed_time(e1) / steps)

        ms_default = timed(lambda: hp.hmat_eval(h, W, Y, q, hp.HMAT_MODE_FP64, stream))
        tune = hp.hmat_autotune(h, q, hp.HMAT_MODE_FP64, stream)
        hp.hmat_profile(h, True)
        for _ in range(20):
            hp.hmat_eval(h, W, Y, q, hp.HMAT_MODE_FP64, stream)
        ph = hp.hmat_phase_times(h)
        hp.hmat_profile(h, False)
        launches = sum(c for _, c in ph.values()) // 20
        ms_eval = timed(lambda: hp.hmat_eval(h, W, Y, q, hp.HMAT_MODE_FP64, stream))
        b = hp.hmat_batch_create([h], hp.HMAT_MODE_FP64)
        try:
            ms_graph = timed(lambda: hp.hmat_batch_eval(b, [W], [Y], stream))
        finally:
            hp.hmat_batch_free(b)
        if hp.hmat_status_poll(h) != hp.HMAT_OK:
            raise RuntimeError("device status error in the HSS steps")
        flops = 2.0 * q * (info["near_values"] + 2 * info["basis_values"] + info["coupling_values"])
        return {"workload": w.name, "n": w.n, "q": q, "mode": "fp64", "levels": info["levels"],
                "sum_rank": info["sum_rank"], "steps": steps, "launches_per_eval": launches,
                "us_per_eval": round(ms_eval * 1e3, 2), "us_per_eval_graph": round(ms_graph * 1e3, 2),
                "us_per_eval_untuned": round(ms_default * 1e3, 2),
                "phases_us_per_eval": {k: round(v[0] / 20 * 1e3, 2) for k, v in ph.items() if v[1]},
                "autotune": tune,
                "value": round(dist.world * q / (ms_eval / 1e3), 1), "unit": "cols/s",
                "gflops": round(flops / (ms_eval / 1e3) / 1e9, 2)}
    finally:
        hp.hmat_free(h)


def run_batch(args, dist) -> dict:
    """Batched mode: 64 independent HMatrices (N log-uniform in [1024, 32768], d 3/8, Gaussian / inverse
    multiquadric, leaf 64-256, tol 1e-5, q uniform in 1..64) evaluated in one CUDA-graph launch, against the
    same evaluations issued one hmat_eval at a time."""
    import torch
    import paper_1812_07152_gb300 as hp
    from workloads import batch_workloads, make_points, normal_rhs
    ws = batch_workloads(64)
    t0 = time.perf_counter()
    handles = [hp.hmat_build(make_points(w), flags=hp.HMAT_LOAD_MIXED, **build_params(w)) for w in ws]
    t_build = time.perf_counter() - t0
    Ws = [torch.from_numpy(normal_rhs(w.n, w.q, w.rhs_seed)).cuda() for w in ws]
    Ys = [torch.empty_like(W) for W in Ws]
    cols = sum(w.q for w in ws)
    stream = torch.cuda.current_stream()
    out = {"matrices": len(ws), "columns_per_step": cols, "n_total": sum(w.n for w in ws),
           "inspector_s": round(t_build, 2), "unit": "cols/s"}

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    for name, mode in (("fp64", hp.HMAT_MODE_FP64), ("mixed", hp.HMAT_MODE_MIXED)):
        b = hp.hmat_batch_create(handles, mode)
        ms_default = dist.max(timed(lambda: hp.hmat_batch_eval(b, Ws, Ys, stream)))
        # autotuned tile shapes per member (bitwise the same results); the next batch call re-captures
        t0 = time.perf_counter()
        for h, w in zip(handles, ws):
            hp.hmat_autotune(h, w.q, mode, stream)
        t_tune = time.perf_counter() - t0
        hp.hmat_batch_free(b)
        b = hp.hmat_batch_create(handles, mode)
        batch_tune = hp.hmat_batch_autotune(b, Ws, Ys, stream)   # the chain grid, on whole replays
        ms_graph = dist.max(timed(lambda: hp.hmat_batch_eval(b, Ws, Ys, stream)))
        info = hp.hmat_batch_info(b)
        ms_loop = dist.max(timed(lambda: [hp.hmat_eval(h, W, Y, W.shape[1], mode, stream)
                                          for h, W, Y in zip(handles, Ws, Ys)]))
        hp.hmat_batch_free(b)
        out[name] = {"value": round(dist.world * cols / (ms_graph / 1e3), 1), "ms_per_step": round(ms_graph, 4),
                     "kernels_per_replay": info["kernels"], "batch_autotune": batch_tune,
                     "untuned_value": round(dist.world * cols / (ms_default / 1e3), 1),
                     "untuned_ms": round(ms_default, 4), "autotune_s": round(t_tune, 2),
                     "one_call_per_matrix_value": round(dist.world * cols / (ms_loop / 1e3), 1),
                     "one_call_per_matrix_ms": round(ms_loop, 4)}
    for h in handles:
        hp.hmat_free(h)
    return out


def run_serving(args, dist) -> dict:
    """Serving mode: resident HMatrices (d = 3 uniform points, Gaussian h = 0.5, tol 1e-6, leaf 256), loaded
    mixed-only (the FP64 blocks dropped), a Poisson stream of requests of q uniform in 1..256 on a random matrix,
    half of them FP32 and half FP64, memory-bounded admission, continuous batching and load shedding (a bounded
    queue: a request that finds it full is refused and counted as dropped); p50/p99 latency from submit to the
    result in pinned host memory, overall and per matrix. After the stream ends (60 s full, 6 s short) the queue
    drains and the run stops."""
    import numpy as np
    import torch
    import paper_1812_07152_gb300 as hp
    from workloads import make_points, serving_workloads
    if args.serve == "full":
        ws, rate, seconds = serving_workloads(), 2000.0, 60.0
    else:
        ws, rate, seconds = serving_workloads((16384, 32768, 65536, 131072)), 1000.0, 6.0
    t0 = time.perf_counter()
    handles = [hp.hmat_build(make_points(w), flags=hp.HMAT_LOAD_MIXED_ONLY, **build_params(w)) for w in ws]
    t_build = time.perf_counter() - t0
    resident = sum(hp.hmat_info(h)["device_bytes"] for h in handles)
    q_max = 256
    rng = np.random.default_rng(7)
    # one pinned W and one pinned Y per matrix and dtype: the requests on a matrix read column slices of its W and
    # write column slices of its Y (concurrent requests overwrite each other's results there: this run measures
    # time, the tests check results)
    Wp = [{dt: torch.from_numpy(rng.standard_normal((w.n, q_max))).to(dt).pin_memory()
           for dt in (torch.float64, torch.float32)} for w in ws]
    Yp = [{dt: torch.empty((w.n, q_max), dtype=dt).pin_memory() for dt in (torch.float64, torch.float32)}
          for w in ws]
    budget = 48 << 30
    max_pending = 16
    sv = hp.hmat_server_create(handles, slots=4, memory_budget=budget, max_q=4 * q_max, mode=hp.HMAT_MODE_MIXED,
                               max_pending=max_pending)
    ids = []
    t_start = time.perf_counter()
    t_next = t_start
    offered = accepted = dropped = cols = 0
    while True:
        t_next += rng.exponential(1.0 / rate)
        if t_next - t_start > seconds:
            break
        now = time.perf_counter()
        if t_next > now:
            time.sleep(t_next - now)
        m = int(rng.integers(0, len(ws)))
        q = int(rng.integers(1, q_max + 1))
        dt = torch.float32 if rng.random() < 0.5 else torch.float64
        offered += 1
        try:
            ids.append(hp.hmat_server_submit(sv, m, Wp[m][dt][:, :q], Yp[m][dt][:, :q]))
        except hp.HmatError as e:
            if e.status != hp.HMAT_EBUSY:
                raise
            dropped += 1
            continue
        accepted += 1
        cols += q
    t_stream = time.perf_counter() - t_start
    failed = sum(hp.hmat_server_wait(sv, rid) != hp.HMAT_OK for rid in ids)
    elapsed = time.perf_counter() - t_start
    st = hp.hmat_server_stats(sv)
    per = [dict(n=w.n, **hp.hmat_server_matrix_stats(sv, i)) for i, w in enumerate(ws)]
    hp.hmat_server_free(sv)
    for h in handles:
        hp.hmat_free(h)
    return {"matrices": [w.n for w in ws], "offered_req_per_s": rate, "seconds": seconds,
            "offered": offered, "served": accepted, "dropped": dropped, "failed": failed,
            "value": round(cols / elapsed, 1), "unit": "cols/s",
            "served_req_per_s": round(accepted / elapsed, 1), "stream_s": round(t_stream, 2),
            "drain_s": round(elapsed - t_stream, 2),
            "p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
            "per_matrix": [{k: (round(v, 3) if isinstance(v, float) else v) for k, v in d.items()} for d in per],
            "requests_per_evaluation": round(st["requests_per_evaluation"], 3),
            "peak_device_bytes": int(st["peak_bytes"]), "resident_bytes": int(resident), "memory_budget": budget,
            "max_pending": max_pending, "slots": 4, "mode": "mixed (FP64 blocks dropped)",
            "dtypes": "half FP32, half FP64 W and Y", "inspector_s": round(t_build, 2)}


def measured_traffic(key: str, near_values: int):
    """DRAM bytes per launch of a kernel, from the ncu capture recorded in profiles/traffic.json,
    scaled by the stored near values; None when the kernel's sources changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[key]
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        if h.hexdigest()[:16] != rec["source_sha256_16"]:
            return None
        return int(rec["dram_bytes_per_near_value"] * near_values)
    except Exception:
        return None


def w_rows(info) -> int:
    return info["n_points"]


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "bf16_tflops": float(p["bf16_tflops"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


# ----------------------------------------------------------------------------- CPU oracle (baseline / reference arm)

def _cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_setup(w):
    from oracle import hmatrix as hm
    t0 = time.perf_counter()
    H, _ = hm.compress_workload(w)
    return hm, H, time.perf_counter() - t0


def _oracle_sample_q(hm, H, w, target_s: float) -> int:
    """Columns per sample so that one oracle evaluation takes about target_s seconds."""
    from workloads import normal_rhs
    q_probe = 4
    t0 = time.perf_counter()
    hm.evaluate(H, normal_rhs(w.n, q_probe, w.rhs_seed))
    t_probe = time.perf_counter() - t0
    q = int(q_probe * target_s / max(t_probe, 1e-3))
    return max(1, min(w.q, q))


def cpu_baseline(w, target_s: float) -> dict:
    from workloads import normal_rhs
    hm, H, t_compress = _oracle_setup(w)
    qs = _oracle_sample_q(hm, H, w, target_s)
    W = normal_rhs(w.n, w.q, w.rhs_seed)[:, :qs].copy()
    t0 = time.perf_counter()
    hm.evaluate(H, W)
    dt = time.perf_counter() - t0
    return {"value": round(qs / dt, 4), "unit": "cols/s", "cores": _cores(), "kind": "oracle",
            "sample": f"FP64 NumPy oracle evaluation of the same HMatrix recipe (oracle-compressed, "
                      f"{t_compress:.0f} s, excluded) on the first {qs} of {w.q} columns of W: {dt:.1f} s"}


def run_reference(args, dist: Dist) -> None:
    if dist.rank != 0:
        return
    from workloads import normal_rhs
    w = workload(args)
    hm, H, t_compress = _oracle_setup(w)
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(args.steps + args.warmup, 1)))
    qs = _oracle_sample_q(hm, H, w, per_step)
    W = normal_rhs(w.n, w.q, w.rhs_seed)[:, :qs].copy()
    for _ in range(args.warmup):
        hm.evaluate(H, W)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        hm.evaluate(H, W)
        times.append(time.perf_counter() - t0)
    mean = sum(times) / len(times)
    value = qs / mean
    sample = (f"FP64 NumPy oracle on the host cores, first {qs} of {w.q} columns per step "
              f"(oracle compression {t_compress:.0f} s excluded)")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "cols/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(mean * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "d": w.d, "q": w.q, "q_sample": qs, "mode": "fp64"},
        "cpu_baseline": {"value": round(value, 4), "unit": "cols/s", "cores": _cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "cols/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    dist = Dist()
    if args.impl == "reference":
        run_reference(args, dist)
    else:
        run_gpu(args, dist)


if __name__ == "__main__":
    main()
