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


def max_over_ranks(ms: float, ws: int, device=None) -> float:
    """The timed region's length as the job sees it: the maximum over ranks
    (every rank holds the same per-GPU workload; no data-path collective)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(bytes_per_step_per_rank: int, steps: int, ms: float, ws: int) -> float:
    """Whole-job algorithmic GB/s: the bytes all ranks processed over the max time."""
    return ws * bytes_per_step_per_rank * steps / (ms * 1e-3) / 1e9


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
    tune = not args.no_autotune

    # ------------------------------------------------------------ buffers
    gen = torch.Generator(device=dev).manual_seed(13010763 + rank)
    # re and im i.i.d. N(0, 1)
    zin = torch.randn(ELEMS, 2, dtype=torch.float32, device=dev, generator=gen).view(torch.complex64).view(ELEMS)
    zout = torch.empty_like(zin)
    t_tune = time.perf_counter()
    plans = {lg: qft.Plan(1 << lg, ELEMS >> lg, autotune=tune, in_place=args.in_place) for lg in logs}
    tune_s = time.perf_counter() - t_tune

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
    for lg in logs:
        plans[lg].time_launches(True)
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
    ms = max_over_ranks(t0.elapsed_time(t1), ws, dev)
    kt = {}
    for lg in logs:
        kt[lg] = plans[lg].launch_times()
        plans[lg].time_launches(False)
    bytes_per_step = 16 * ELEMS * len(logs)
    flops_per_step = sum(5 * ELEMS * lg for lg in logs)
    value = job_value(bytes_per_step, args.steps, ms, ws)
    gflops = ws * flops_per_step * args.steps / (ms * 1e-3) / 1e9
    per_size = {}
    for lg in logs:
        times = [e[0].elapsed_time(e[1]) for e in evs[lg]]
        per_size[lg] = sum(times) / len(times)
    peak, peak_src = measured_peaks()
    comp_j = {lg: plans[lg].comp_classes() for lg in logs}
    roof, kernel_share = roofline(kt, peak, peak_src, comp_j)
    launches = sum(n for lg in logs for (_, n) in kt[lg].values())
    # the path's own fraction: the method's 16 N bytes per transform over the step
    roof["path_achieved"] = round(value, 1)
    roof["path_frac"] = round(value / peak, 4)
    # HBM passes per execute: every launch of the path reads and writes each
    # element's 8-byte cell once (the C/S table launches of the large-row path
    # move less and are counted as passes, so this is an upper estimate); the
    # ncu capture of the NODE kernel measured 0.98 of its pass bytes
    def passes(lg):
        launches = sum(n for (_, n) in kt[lg].values()) / args.steps
        cr = plans[lg].schedule()["chunk_rows"]
        chunks = -(-(ELEMS >> lg) // cr) if cr > 0 else 1
        return round(launches / chunks, 2)
    roof["traffic_ratio_est"] = {f"2^{lg}": passes(lg) for lg in logs}

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
    schedules = {f"2^{lg}": plans[lg].schedule() for lg in logs}
    comp = {f"2^{lg}": comp_j[lg] for lg in logs}
    scratch = {f"2^{lg}": plans[lg].scratch_bytes() for lg in logs}

    # ------------------------------------------------------------- e2e
    e2e = None
    if not args.no_e2e:
        del zout
        e2e = run_e2e(args, logs, dev, stream, torch, qft, tune)
    zin = zout = None
    plans = None
    torch.cuda.empty_cache()

    extras = None
    if not args.no_extras and rank == 0:
        extras = run_extras(args, dev, stream, torch, qft, orc, tune, peak)
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        gbs, t_step, rows = cpu_reference_run(logs, 1, 0, args.ref_sample_elems, threads)
        cpu = {"value": round(gbs, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
               "sample": "FP64 oracle, one pass over rows per size " +
                         ", ".join(f"2^{lg}:{rows[lg]}" for lg in logs)}

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "batched-2^28 complex64 forward, N in " +
                           ",".join(f"2^{l}" for l in logs), "elements_per_size": ELEMS,
                           "sizes_not_yet_supported": [f"2^{l}" for l in CONFIG_LOGS if l not in logs],
                           "l2": "inputs (2 GiB) larger than L2, no flush",
                           "schedules": schedules, "autotune": tune, "autotune_s": round(tune_s, 2),
                           "compensated_classes": comp,
                           "large_row_scratch": "one copy (in-place backward levels)" if args.in_place
                           else "two copies",
                           "scratch_bytes": scratch},
                "gflops_5nlog2n": round(gflops, 1),
                "frac_of_hbm": round(value / peak, 4),
                "rel_err_vs_fp64": {"max": err_max, "mean": float(np.nanmean(err_mean)) if len(err_mean) > 1 else None, "rows": len(err_mean) - 1},
                "per_size_ms": {f"2^{lg}": round(per_size[lg], 4) for lg in logs},
                "per_size_gbs": {f"2^{lg}": round(16 * ELEMS / (per_size[lg] * 1e-3) / 1e9, 1) for lg in logs},
                "kernel_ms_per_step": kernel_share(args.steps),
                "roofline": roof,
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches, "extras": extras}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# dram__bytes_read.sum + dram__bytes_write.sum per launch of a kernel, from one
# ncu capture of the named kernel at the stated size (scaled to a launch over
# 2^28 elements by the rows, since the traffic grows in proportion to them);
# None once the kernel has changed since the capture.
NCU_TRAFFIC = {("k_large_node", 18): 465741824 * 16}   # N = 2^18 capture: 465.7 MB over 2^24 elements, x 16
ROOF_SIZE = {"k_large_node": 18}                         # the size the roofline line reports for that kernel


def comp_factor(J):
    """Bytes per element per pass of the large-row kernels over the 16 B of the
    plain cells: the compensated classes (the share 1 - 2^-J of the cells) also
    move their lo parts."""
    return 2.0 - 2.0 ** (-J) if J > 0 else 1.0


def roofline(kt, peak, peak_src, comp=None):
    """Roofline of the kernel with the largest summed time over the timed
    region.  Every launch of every kernel of the path reads and writes each of
    the 2^28 elements' 8-byte cells once (row kernel: the transform's 8N in +
    8N out; large-row kernels: 8N of class data in and 8N out per pass), plus
    the lo parts of the compensated classes' cells, so its algorithmic bytes
    per launch are 16 * 2^28 * comp_factor(J) (one launch per size at this
    workload).  `achieved` is for the size in ROOF_SIZE (the ncu capture's),
    `per_size` for every size the kernel ran at."""
    comp = comp or {}
    tot = {}
    for lg, d in kt.items():
        for k, (ms, n) in d.items():
            tot[k] = tot.get(k, 0.0) + ms
    dom = max(tot, key=tot.get)
    sizes = sorted(lg for lg in kt if dom in kt[lg])
    per_size = {}
    for lg in sizes:
        ms, n = kt[lg][dom]
        bpl = 16 * ELEMS * comp_factor(comp.get(lg, 0))
        per_size[f"2^{lg}"] = {"gbs": round(bpl / (ms / n * 1e-3) / 1e9, 1), "avg_launch_ms": round(ms / n, 4),
                               "launches": n, "bytes_per_launch": int(bpl), "compensated_classes": comp.get(lg, 0)}
    lg0 = ROOF_SIZE.get(dom, sizes[-1])
    if lg0 not in sizes:
        lg0 = sizes[-1]
    ms, n = kt[lg0][dom]
    bpl = 16 * ELEMS * comp_factor(comp.get(lg0, 0))
    avg = ms / n
    achieved = bpl / (avg * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "size": f"2^{lg0}",
            "achieved": round(achieved, 1), "peak": peak, "peak_source": peak_src, "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "frac_basis": "this kernel's own bytes per launch at this size: 16 B per element per pass, x (2 - 2^-J) "
                          "with J compensated classes (row kernel: the transform's input and output; large-row "
                          "kernels: scratch to scratch)",
            "traffic": NCU_TRAFFIC.get((dom, lg0)),
            "bytes_per_launch": int(bpl), "launches": n, "avg_launch_ms": round(avg, 4), "per_size": per_size}

    def share(steps):
        return {k: round(v / steps, 3) for k, v in sorted(tot.items(), key=lambda x: -x[1])}
    return roof, share


def run_e2e(args, logs, dev, stream, torch, qft, tune):
    """Same metric through the public API with host buffers: every step copies
    each size's input (2 GiB) from pinned host memory, transforms it and copies
    the spectrum back (qft.fft_host: chunks, copies overlapped with the
    transforms)."""
    qft.set_autotune(tune)
    host_in = torch.randn(ELEMS, dtype=torch.complex64).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    steps = max(1, min(args.steps, 3))

    ins = [host_in.view(ELEMS // (1 << lg), 1 << lg) for lg in logs]
    outs = [host_out.view(ELEMS // (1 << lg), 1 << lg) for lg in logs]

    def one():   # one call: the copies of one size overlap the transforms of the next
        qft.fft_host(ins, outs)
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
    nbytes = 16 * ELEMS * len(logs)
    qft.set_autotune(False)
    return {"value": round(nbytes / (ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": 8 * ELEMS * len(logs), "d2h_bytes_per_step": 8 * ELEMS * len(logs),
            "ms_per_step": round(ms, 3),
            "workload": "the same sizes and batches, one qft.fft_host() call over the sizes' pinned host "
                        "tensors (chunked; copies in and out overlap the transforms on three streams), "
                        "copies included"}


def _time(fn, torch, stream, reps=3, warm=2):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _rel_errs(Y, ref):
    e = np.linalg.norm(Y - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    return {"max": float(e.max()), "mean": float(e.mean()), "rms": float(np.sqrt(np.mean(e * e)))}


def run_extras(args, dev, stream, torch, qft, orc, tune, peak):
    """The other measured forms of the path: single small transform, inverse,
    real input, uneven batch, FP16/BF16 storage, spectral filter, 2^24."""
    from paper_1301_0763_gb300 import inputs
    ex = {}
    gen = torch.Generator(device=dev).manual_seed(13010763 + 7)

    # ---- N = 1024, batch 64 (latency) and N = 2^10 x 2^18 (bandwidth)
    x = torch.from_numpy(inputs.uniform_complex(64, 1024, seed=1)).to(dev)
    y = torch.empty_like(x)
    p = qft.Plan(1024, 64, autotune=tune)
    us_plain = 1e3 * _time(lambda: p.execute(qft.OP_FORWARD, x, y), torch, stream, reps=200, warm=10)
    c1 = {"us_per_execute": round(us_plain, 2)}
    try:
        gs = torch.cuda.Stream()
        gs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(gs):
            p.execute(qft.OP_FORWARD, x, y)
        torch.cuda.current_stream().wait_stream(gs)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            p.execute(qft.OP_FORWARD, x, y)
        c1["us_graph_replay"] = round(1e3 * _time(graph.replay, torch, stream, reps=200, warm=10), 2)
    except Exception as exc:  # noqa: BLE001  (report, do not fail the bench)
        c1["graph_error"] = str(exc)[:200]
    torch.cuda.synchronize()
    ref = orc.cdft(x.cpu().numpy())
    c1["rel_err_vs_fp64"] = _rel_errs(y.cpu().numpy().astype(np.complex128), ref)
    z = torch.randn(1 << 28, 2, device=dev, generator=gen).view(torch.complex64).view(1 << 18, 1 << 10)
    zo = torch.empty_like(z)
    pb = qft.Plan(1 << 10, 1 << 18, autotune=tune)
    ms = _time(lambda: pb.execute(qft.OP_FORWARD, z, zo), torch, stream)
    c1["n1024_batch2^18_gbs"] = round(16 * (1 << 28) / (ms * 1e-3) / 1e9, 1)
    ex["n1024"] = c1

    # ---- inverse and real input at the batched sizes
    inv, real = {}, {}
    zv = z.view(-1)
    for lg in CONFIG_LOGS:
        N = 1 << lg
        a, b = zv.view(-1, N), zo.view(-1, N)
        pl = qft.Plan(N, a.shape[0], autotune=tune)
        ms = _time(lambda: pl.execute(qft.OP_INVERSE, a, b), torch, stream)
        inv[f"2^{lg}"] = round(16 * (1 << 28) / (ms * 1e-3) / 1e9, 1)
        pl.destroy()
        xr = zv.view(torch.float32)[: 1 << 28].view(-1, N)
        yr = zo.view(-1)[: (xr.shape[0] * (N // 2 + 1))].view(xr.shape[0], N // 2 + 1)
        pr = qft.Plan(N, xr.shape[0], kind=qft.KIND_R2C, autotune=tune)
        ms = _time(lambda: pr.execute(qft.OP_FORWARD, xr, yr), torch, stream)
        real[f"2^{lg}"] = round(xr.shape[0] * (4 * N + 8 * (N // 2 + 1)) / (ms * 1e-3) / 1e9, 1)
        pr.destroy()
    ex["inverse_gbs"] = inv
    ex["real_forward_gbs"] = real
    # the cost of the compensated classes: the same forward with every class
    # tree in plain FP32 (QFT_PLAN_FP32_PLAIN), and its error on sampled rows
    plain = {}
    for lg in [l for l in CONFIG_LOGS if l >= 16]:
        N = 1 << lg
        a, b = zv.view(-1, N), zo.view(-1, N)
        pl = qft.Plan(N, a.shape[0], autotune=tune, plain=True)
        ms = _time(lambda: pl.execute(qft.OP_FORWARD, a, b), torch, stream)
        torch.cuda.synchronize()
        rows = [0, a.shape[0] // 2, a.shape[0] - 1]
        e = _rel_errs(b[rows].cpu().numpy().astype(np.complex128), orc.cdft(a[rows].cpu().numpy()))
        plain[f"2^{lg}"] = {"gbs": round(16 * (1 << 28) / (ms * 1e-3) / 1e9, 1), "rel_err_vs_fp64_max": e["max"],
                            "comp_classes": 0}
        pl.destroy()
    ex["fp32_plain_forward"] = plain
    # standalone DCT-0 / DST-0 (eqs qft_0B, qft_0C): 2^28 reals in and out per size
    r2r = {}
    for lg in (12, 16, 20):
        N = 1 << lg
        for name, kind, L in (("dct0", qft.KIND_DCT0, N // 2 + 1), ("dst0", qft.KIND_DST0, N // 2 - 1)):
            rows = (1 << 28) // L
            xr = zv.view(torch.float32)[: rows * L].view(rows, L)
            yr = zo.view(-1).view(torch.float32)[: rows * L].view(rows, L)
            pr = qft.Plan(N, rows, kind=kind, autotune=tune)
            ms = _time(lambda: pr.execute(qft.OP_FORWARD, xr, yr), torch, stream)
            r2r[f"{name}_2^{lg}"] = round(8 * rows * L / (ms * 1e-3) / 1e9, 1)
            pr.destroy()
    ex["dct0_dst0_gbs"] = r2r
    del z, zo, zv
    torch.cuda.empty_cache()

    # ---- uneven batch: one graph launch against a per-length loop
    log2n = inputs.ragged_log2n(4096, seed=2)
    off = inputs.ragged_offsets(log2n)
    total = int(off[-1])
    zr = torch.randn(total, 2, device=dev, generator=gen).view(torch.complex64).view(total)
    yr = torch.empty_like(zr)
    t_plan = time.perf_counter()
    rp = qft.RaggedPlan(off, log2n, autotune=tune)
    t_plan = time.perf_counter() - t_plan
    ms_graph = _time(lambda: rp.execute(qft.OP_FORWARD, zr, yr), torch, stream)
    # the same rows sorted by length into contiguous per-length buffers
    order = np.argsort(log2n, kind="stable")
    lens = np.left_shift(1, log2n[order].astype(np.int64))
    classes = sorted(set(log2n.tolist()))
    bufs, loop_plans, pos = [], [], 0
    for r in classes:
        cnt = int((log2n == r).sum())
        n = cnt << r
        bufs.append((zr[pos:pos + n].view(cnt, 1 << r), yr[pos:pos + n].view(cnt, 1 << r)))
        loop_plans.append(qft.Plan(1 << r, cnt, autotune=tune))
        pos += n
    assert pos == total and int(lens.sum()) == total

    def loop():
        for pl, (a, b) in zip(loop_plans, bufs):
            pl.execute(qft.OP_FORWARD, a, b)
    ms_loop = _time(loop, torch, stream)
    nbytes = 16 * total
    ex["ragged_4096"] = {"total_complex": total, "classes": len(classes), "graph_ms": round(ms_graph, 3),
                         "loop_ms": round(ms_loop, 3), "graph_gbs": round(nbytes / (ms_graph * 1e-3) / 1e9, 1),
                         "loop_gbs": round(nbytes / (ms_loop * 1e-3) / 1e9, 1),
                         "graph_speedup": round(ms_loop / ms_graph, 3), "plan_s": round(t_plan, 2),
                         "loop": "one plain plan per length over the rows sorted by length"}
    rp.destroy()
    for pl in loop_plans:
        pl.destroy()
    del zr, yr, bufs
    torch.cuda.empty_cache()

    # ---- FP16 / BF16 storage
    half = {}
    for name, dt, code in (("fp16", torch.float16, qft.DTYPE_F16), ("bf16", torch.bfloat16, qft.DTYPE_BF16)):
        for lg in (10, 13, 16):
            N, B = 1 << lg, 1 << 14
            xh = (torch.rand(B, N, 2, device=dev, generator=gen) * 2 - 1).to(dt)
            yh = torch.empty_like(xh)
            ph = qft.Plan(N, B, dtype=code, autotune=tune)
            ms = _time(lambda: ph.execute(qft.OP_FORWARD, xh, yh), torch, stream)
            ent = {"gbs": round(8 * N * B / (ms * 1e-3) / 1e9, 1)}
            ph.destroy()
            del xh, yh
            rows = 32
            ps = qft.Plan(N, rows, dtype=code)
            pf = qft.Plan(N, rows)
            for setname, z64 in (("uniform", inputs.uniform_complex(rows, N, seed=4, dtype=np.complex128)),
                                 ("student_t3", inputs.student_t_complex(rows, N, seed=4))):
                pair = torch.from_numpy(np.stack([z64.real, z64.imag], -1))
                xs = pair.to(dt).to(dev)
                ys = torch.empty_like(xs)
                ps.execute(qft.OP_FORWARD, xs, ys)
                torch.cuda.synchronize()
                xr64 = xs.float().cpu().numpy().astype(np.float64)
                xr64 = xr64[..., 0] + 1j * xr64[..., 1]
                Y = ys.float().cpu().numpy().astype(np.float64)
                Y = Y[..., 0] + 1j * Y[..., 1]
                ref_a = orc.cdft(xr64)
                ref_b = orc.cdft(z64)
                x32 = torch.from_numpy(z64.astype(np.complex64)).to(dev)
                y32 = torch.empty_like(x32)
                pf.execute(qft.OP_FORWARD, x32, y32)
                torch.cuda.synchronize()
                ref_32 = orc.cdft(x32.cpu().numpy())
                ent[setname] = {"vs_oracle_of_rounded_input": _rel_errs(Y, ref_a),
                                "vs_oracle_of_fp64_input": _rel_errs(Y, ref_b),
                                "fp32_path_vs_oracle": _rel_errs(y32.cpu().numpy().astype(np.complex128), ref_32),
                                "rows": rows}
            ps.destroy()
            pf.destroy()
            half[f"{name}_2^{lg}"] = ent
    ex["half_storage"] = half
    torch.cuda.empty_cache()

    # ---- fixed-point variant: int16 Q15 in, int32 block floating point out;
    # 2^26 samples per size, bytes 4N in + 8N + 4 out per row
    fx = {}
    for lg in (6, 10, 12, 13):
        N = 1 << lg
        rows = (1 << 26) // N
        zq = torch.randint(-32768, 32768, (rows, N, 2), device=dev, dtype=torch.int32, generator=gen).to(torch.int16)
        Xq = torch.empty((rows, N, 2), dtype=torch.int32, device=dev)
        Eq = torch.empty(rows, dtype=torch.int32, device=dev)
        pq = qft.Plan(N, rows, dtype=qft.DTYPE_I16)
        ms = _time(lambda: pq.execute_fixed(zq, Xq, Eq), torch, stream)
        torch.cuda.synchronize()
        pick = [0, rows // 3, rows - 1]
        zs = zq[pick].cpu().numpy()
        Xo, Eo = orc.cdft_fx(zs)
        same = bool(np.array_equal(Xq[pick].cpu().numpy(), Xo) and np.array_equal(Eq[pick].cpu().numpy(), Eo))
        zf = (zs[..., 0] + 1j * zs[..., 1]) / 2.0 ** 15
        e = _rel_errs(orc.fx_value(Xo, Eo), np.fft.fft(zf.astype(np.complex128), axis=-1))
        fx[f"2^{lg}"] = {"gbs": round(rows * (12 * N + 4) / (ms * 1e-3) / 1e9, 1), "ms": round(ms, 4),
                         "bit_exact_sampled_rows": same, "rel_err_vs_fp64_max": e["max"]}
        pq.destroy()
        del zq, Xq, Eq
    ex["fixed_point"] = fx
    torch.cuda.empty_cache()

    # ---- spectral filter y = irfft(W * rfft(x)), x [64, 64, 4096]
    B, C, N = 64, 64, 4096
    xf = torch.randn(B, C, N, device=dev, generator=gen)
    W = (0.02 * torch.randn(C, N // 2 + 1, 2, device=dev, generator=gen)).view(torch.complex64).view(C, N // 2 + 1)
    yf = torch.empty_like(xf)
    gx = torch.empty_like(xf)
    gW = torch.empty_like(W)
    fp = qft.FilterPlan(N, B, C)
    ms_f = _time(lambda: fp.forward(xf, W, yf), torch, stream, reps=10)
    ms_b = _time(lambda: fp.backward(xf, W, yf, gx, gW), torch, stream, reps=10)
    rowb = B * C * N * 4
    ex["spectral_filter"] = {"forward_ms": round(ms_f, 4), "backward_ms": round(ms_b, 4),
                             "forward_gbs": round((2 * rowb + W.numel() * 8) / (ms_f * 1e-3) / 1e9, 1),
                             "backward_gbs": round((3 * rowb + 2 * W.numel() * 8) / (ms_b * 1e-3) / 1e9, 1),
                             "bytes": "forward x + y + W; backward x + gy + gx + W + gW"}
    fp.destroy()
    del xf, yf, gx, gW, W
    torch.cuda.empty_cache()

    # ---- one N = 2^24 transform, forward and backward
    N = 1 << 24
    x = torch.randn(N, 2, device=dev, generator=gen).view(torch.complex64).view(1, N)
    y = torch.empty_like(x)
    g2 = torch.empty_like(x)
    pl = qft.Plan(N, 1, autotune=tune)
    pl.time_launches(True)
    ms_f = _time(lambda: pl.execute(qft.OP_FORWARD, x, y), torch, stream, reps=3, warm=0)
    kt = pl.launch_times()
    ms_b = _time(lambda: pl.execute(qft.OP_FORWARD_ADJOINT, y, g2), torch, stream, reps=3, warm=0)
    pl.time_launches(False)
    launches = sum(n for (_, n) in kt.values()) // 3
    ex["n2^24"] = {"forward_ms": round(ms_f, 3), "backward_ms": round(ms_b, 3),
                   "forward_gbs": round(16 * N / (ms_f * 1e-3) / 1e9, 1),
                   "launches_per_execute": launches,
                   "bytes_moved_per_execute_est": 16 * N * launches,
                   "schedule": pl.schedule()}
    pl.destroy()
    return ex


def run_fixed_only(args):
    """The fixed-point variant alone at one length (a profiling run): `warmup`
    untimed and `steps` timed executes over 2^26 Q15 samples; one JSON line."""
    import torch
    from paper_1301_0763_gb300 import build, qft
    build.build()
    qft.load_library()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    N = 1 << args.fixed
    rows = (1 << 26) // N
    gen = torch.Generator(device=dev).manual_seed(13010763 + 8)
    zq = torch.randint(-32768, 32768, (rows, N, 2), device=dev, dtype=torch.int32, generator=gen).to(torch.int16)
    X = torch.empty((rows, N, 2), dtype=torch.int32, device=dev)
    E = torch.empty(rows, dtype=torch.int32, device=dev)
    p = qft.Plan(N, rows, dtype=qft.DTYPE_I16)
    stream = torch.cuda.current_stream()
    ms = _time(lambda: p.execute_fixed(zq, X, E), torch, stream, reps=max(1, args.steps), warm=max(1, args.warmup))
    print(json.dumps({"workload": f"fixed-point forward, N = 2^{args.fixed}, {rows} rows", "ms": round(ms, 4),
                      "gbs": round(rows * (12 * N + 4) / (ms * 1e-3) / 1e9, 1), "launches": args.steps + args.warmup}))


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
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads (profiling runs)")
    ap.add_argument("--no-autotune", action="store_true", help="default schedules instead of autotuned ones")
    ap.add_argument("--in-place", action="store_true",
                    help="large rows on the one-scratch schedule (QFT_PLAN_IN_PLACE)")
    ap.add_argument("--sizes", default="", help="comma-separated log2 N subset (profiling runs)")
    ap.add_argument("--elems-log2", type=int, default=28,
                    help="complex elements per size (28 = the benchmark; smaller for profiler captures)")
    ap.add_argument("--fixed", type=int, default=0, metavar="LG",
                    help="profiling runs: time only the fixed-point variant at N = 2^LG (2^26 samples)")
    args = ap.parse_args()
    global SIZES_OVERRIDE, ELEMS
    ELEMS = 1 << args.elems_log2
    if args.sizes:
        SIZES_OVERRIDE = [int(v) for v in args.sizes.split(",")]
    if args.impl == "reference":
        run_reference(args)
    elif args.fixed:
        run_fixed_only(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
