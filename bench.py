"""Benchmark of the GB300 improved-QFT library on the batched-transform workload.

Workload ("batched-2^28"): complex64 rows with i.i.d. standard-normal re and im,
N in {2^12, 2^14, 2^16, 2^18, 2^20} with batch = 2^28 / N, i.e. 2 GiB in and
2 GiB out per size.  One step = the forward transform of every size this
build supports, one launch per size.  Inputs (2 GiB) are larger than the
129 MB L2, so no flush is needed between launches.

Metric: algorithmic HBM bytes per second (16 N bytes per complex transform:
read 8 N + write 8 N), also reported as 5 N log2 N GFLOP/s and as a fraction
of the measured HBM copy bandwidth; plus the relative error of sampled rows
against the FP64 oracle.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs the same per-GPU workload (weak
scaling, no collective on the data path); the timed region is bracketed by
barriers and the max over ranks is reported by rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CONFIG_LOGS = [12, 14, 16, 18, 20]
ELEMS = 1 << 28
METRIC = "FP32 batched FFT GB/s & 5Nlog2N GFLOP/s vs HBM roofline; rel err vs FP64"


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
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
        except subprocess.TimeoutExpired:
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
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_reference_run(logs, steps, warmup, sample_elems, threads):
    """Times the FP64 oracle (as it stands) on a bounded sample of each size."""
    from oracle import oracle as orc
    from paper_1301_0763_gb300 import inputs
    data = {}
    for lg in logs:
        N = 1 << lg
        rows = max(1, sample_elems // N)
        data[lg] = inputs.normal_complex(rows, N, seed=1)
    def one_step():
        t0 = time.perf_counter()
        nbytes = 0
        for lg in logs:
            z = data[lg]
            orc.cdft(z, threads=threads)
            nbytes += 16 * z.size
        return time.perf_counter() - t0, nbytes
    for _ in range(warmup):
        one_step()
    tot_t, tot_b = 0.0, 0
    for _ in range(steps):
        t, b = one_step()
        tot_t += t
        tot_b += b
    return tot_b / tot_t / 1e9, tot_t / max(steps, 1), {lg: data[lg].shape[0] for lg in logs}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    logs = supported_logs()
    sample = args.ref_sample_elems
    gbs, t_step, rows = cpu_reference_run(logs, args.steps, args.warmup, sample, threads)
    desc = "FP64 oracle, rows per size " + ", ".join(f"2^{lg}:{rows[lg]}" for lg in logs)
    line = {"impl": "reference", "metric": METRIC, "value": round(gbs, 4), "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t_step * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batched-2^28 complex64, N in " + ",".join(f"2^{l}" for l in logs) +
                       " (bounded sample per step)", "elements_per_size": ELEMS,
                       "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": round(gbs, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": round(gbs, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SIZES_OVERRIDE = None


def supported_logs():
    from paper_1301_0763_gb300 import qft  # noqa: F401  (library must load)
    logs = list(CONFIG_LOGS)
    if SIZES_OVERRIDE:
        logs = [lg for lg in SIZES_OVERRIDE if lg in logs]
    return logs


def run_gpu(args):
    import torch
    from paper_1301_0763_gb300 import build, qft
    from oracle import oracle as orc

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    qft.load_library()
    logs = supported_logs()
    stream = torch.cuda.current_stream()

    # ------------------------------------------------------------ buffers
    gen = torch.Generator(device=dev).manual_seed(13010763 + rank)
    # re and im i.i.d. N(0, 1)
    zin = torch.randn(ELEMS, 2, dtype=torch.float32, device=dev, generator=gen).view(torch.complex64).view(ELEMS)
    zout = torch.empty_like(zin)
    plans = {lg: qft.Plan(1 << lg, ELEMS >> lg) for lg in logs}

    def step(evs=None):
        for lg in logs:
            N = 1 << lg
            a = zin.view(ELEMS // N, N)
            b = zout.view(ELEMS // N, N)
            if evs is not None:
                evs[lg][0].record(stream)
            plans[lg].execute(qft.OP_FORWARD, a, b, stream)
            if evs is not None:
                evs[lg][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()

    evs = {lg: [[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
                for _ in range(args.steps)] for lg in logs}
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s in range(args.steps):
        step({lg: evs[lg][s] for lg in logs})
    t1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = t0.elapsed_time(t1)
    if ws > 1:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    bytes_per_step = 16 * ELEMS * len(logs)
    flops_per_step = sum(5 * ELEMS * lg for lg in logs)
    value = ws * bytes_per_step * args.steps / (ms * 1e-3) / 1e9
    gflops = ws * flops_per_step * args.steps / (ms * 1e-3) / 1e9
    per_size = {}
    for lg in logs:
        times = [e[0].elapsed_time(e[1]) for e in evs[lg]]
        per_size[lg] = sum(times) / len(times)
    dom = max(per_size, key=per_size.get)
    peak, peak_src = measured_peaks()
    achieved = 16 * ELEMS / (per_size[dom] * 1e-3) / 1e9

    # ------------------------------------------------------- accuracy sample
    err_max, err_mean = 0.0, [float("nan")]
    g = np.random.default_rng(5)
    for lg in ([] if args.no_accuracy else logs):
        N = 1 << lg
        rows = ELEMS // N
        idx = np.unique(np.concatenate([[0, rows - 1], g.integers(0, rows, 6)]))
        plans[lg].execute(qft.OP_FORWARD, zin.view(rows, N), zout.view(rows, N), stream)
        torch.cuda.synchronize()
        zs = zin.view(rows, N)[idx].cpu().numpy()
        Xs = zout.view(rows, N)[idx].cpu().numpy().astype(np.complex128)
        ref = orc.cdft(zs)
        e = np.linalg.norm(Xs - ref, axis=1) / np.linalg.norm(ref, axis=1)
        err_max = max(err_max, float(e.max()))
        err_mean += e.tolist()

    # ------------------------------------------------------------- e2e
    e2e = None if args.no_e2e else run_e2e(args, logs, dev, stream, torch, qft)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        gbs, t_step, rows = cpu_reference_run(logs, 1, 0, args.ref_sample_elems, threads)
        cpu = {"value": round(gbs, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
               "sample": "FP64 oracle, one pass over rows per size " +
                         ", ".join(f"2^{lg}:{rows[lg]}" for lg in logs)}

    info = plans[dom].info()
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "batched-2^28 complex64 forward, N in " +
                           ",".join(f"2^{l}" for l in logs), "elements_per_size": ELEMS,
                           "sizes_not_yet_supported": [f"2^{l}" for l in CONFIG_LOGS if l not in logs],
                           "l2": "inputs (2 GiB) larger than L2, no flush",
                           "threads_per_cta": info["threads"], "ctas": info["ctas"]},
                "gflops_5nlog2n": round(gflops, 1),
                "frac_of_hbm": round(value / peak, 4),
                "rel_err_vs_fp64": {"max": err_max, "mean": float(np.nanmean(err_mean)) if len(err_mean) > 1 else None, "rows": len(err_mean) - 1},
                "per_size_ms": {f"2^{lg}": round(per_size[lg], 4) for lg in logs},
                "per_size_gbs": {f"2^{lg}": round(16 * ELEMS / (per_size[lg] * 1e-3) / 1e9, 1) for lg in logs},
                "roofline": {"bound": "hbm", "kernel": f"k_rows C2C f32 (N=2^{dom})",
                             "achieved": round(achieved, 1), "peak": peak, "peak_source": peak_src,
                             "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None},
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": args.steps * len(logs)}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_e2e(args, logs, dev, stream, torch, qft):
    """Same metric through the public API with host buffers: every step copies
    its input from pinned host memory, transforms, and copies the spectrum back."""
    lg = logs[0]
    N = 1 << lg
    rows = ELEMS // N
    host_in = torch.randn(rows, N, dtype=torch.complex64).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    steps = max(1, min(args.steps, 3))
    def one():
        d = host_in.to(dev, non_blocking=True)
        X = qft.fft(d)
        host_out.copy_(X, non_blocking=True)
    one()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        one()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    nbytes = 16 * ELEMS
    return {"value": round(nbytes / (ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": 8 * ELEMS, "d2h_bytes_per_step": 8 * ELEMS,
            "workload": f"N=2^{lg}, batch {rows}, fft() on pinned host data"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-sample-elems", type=int, default=1 << 24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--sizes", default="", help="comma-separated log2 N subset (profiling runs)")
    ap.add_argument("--elems-log2", type=int, default=28,
                    help="complex elements per size (28 = the benchmark; smaller for profiler captures)")
    args = ap.parse_args()
    global SIZES_OVERRIDE, ELEMS
    ELEMS = 1 << args.elems_log2
    if args.sizes:
        SIZES_OVERRIDE = [int(v) for v in args.sizes.split(",")]
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
