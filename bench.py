"""ST-HOSVD throughput benchmark (input GB/s) on GB300.

One step = one whole ST-HOSVD (Algorithm 1: norm, then per mode Gram,
eigensolve, rank cut, TTM) of one synthetic tensor already resident in HBM,
through the library's C ABI.  Default workload: the 5-way 500x500x500x11x8
FP32 tensor (44 GB, core 60x60x60x11x6 with decay 10^(-0.08 sum idx),
relative noise 1e-7, eps = 1e-4).  The input is larger than L2, so no L2
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec mixed|fp32|fp64]
  python bench.py --impl reference      # the FP64 CPU oracle on host cores

Prints one JSON line (rank 0).  N > 1 runs N independent replicas, one per
GPU (the path has no cross-GPU exchange): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
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

METRIC = "ST-HOSVD input GB/s at eps=1e-4, mixed vs FP64 path; Gram/TTM % of roofline"

WORKLOADS = {
    # recon: the subtensor [0, end) rebuilt by multi-TTM in every step
    "large": dict(dims=(500, 500, 500, 11, 8), core=(60, 60, 60, 11, 6), decay=0.08, eta=1e-7,
                  eps=1e-4, dtype="f32", recon=(500, 500, 500, 11, 1)),
    "c256": dict(dims=(256, 256, 256, 11, 32), core=(40, 40, 40, 11, 16), decay=0.1, eta=1e-7,
                 eps=1e-4, dtype="f32", recon=(256, 256, 256, 11, 1)),
    "c200": dict(dims=(200, 200, 200, 50), core=(30, 30, 30, 12), decay=0.15, eta=1e-6,
                 eps=1e-4, dtype="f64", recon=(200, 200, 200, 1)),
    "small": dict(dims=(40, 50, 30), core=(5, 6, 4), decay=0.0, eta=1e-4, eps=1e-3, dtype="f64",
                  recon=(40, 50, 30)),
    # 64 tensors of uneven shapes compressed by one batched call per step:
    # 3-way cubes with sides uniform in [48, 256] and 4-way tensors
    # [32..160]^3 x [4..16], FP32, core sides 8-32, decay 10^(-0.2 sum idx),
    # relative noise 1e-6
    "batch64": dict(batch=64, decay=0.2, eta=1e-6, eps=1e-4, dtype="f32"),
    # the large workload's first two time steps and 40 of its 500 mode-2
    # slices: a 0.9 GB case of the same kernels for profiler captures
    "prof": dict(dims=(500, 500, 40, 11, 2), core=(60, 60, 40, 11, 2), decay=0.08, eta=1e-7,
                 eps=1e-4, dtype="f32", recon=(500, 500, 40, 11, 1)),
    # a 2.2 GB case whose mode-1 view has the large workload's row-mode shape
    # (L = R_0 ~ 54, I = 500, more than 4096 slabs: the uncompensated kernel)
    "prof_row": dict(dims=(256, 500, 32, 11, 12), core=(60, 60, 32, 11, 12), decay=0.08, eta=1e-7,
                     eps=1e-4, dtype="f32", recon=(256, 500, 32, 11, 1)),
}

FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x 2 x max clock


def peaks():
    p = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "src": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        p.update({k: float(m[k]) for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained")})
        p["src"] = "measured"
    except Exception:
        pass
    return p


def batch_shapes(w, seed):
    """(dims, core) of every tensor of a batched workload (seeded)."""
    rng = np.random.default_rng(1000 + seed)
    out = []
    for k in range(w["batch"]):
        if k % 2 == 0:
            a = int(rng.integers(48, 257))
            dims = (a, a, a)
        else:
            dims = tuple(int(v) for v in rng.integers(32, 161, size=3)) + (int(rng.integers(4, 17)),)
        core = tuple(min(d, int(rng.integers(8, 33))) for d in dims)
        out.append((dims, core))
    return out


def describe(w):
    if "batch" in w:
        return (f"{w['batch']} {w['dtype']} tensors: 3-way cubes, sides uniform in [48, 256], and "
                f"4-way [32..160]^3 x [4..16], cores 8-32 per side, decay 10^(-{w['decay']}*sum idx), "
                f"noise {w['eta']:g}, eps {w['eps']:g}")
    d = "x".join(map(str, w["dims"]))
    c = "x".join(map(str, w["core"]))
    gb = np.prod(w["dims"]) * (4 if w["dtype"] == "f32" else 8) / 1e9
    return (f"{d} {w['dtype']} ({gb:.1f} GB), core {c}, decay 10^(-{w['decay']}*sum idx), "
            f"noise {w['eta']:g}, eps {w['eps']:g}, mode order 0..N-1")


# ------------------------------------------------------------- clocks

class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.p = None
        self.idx = gpu_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
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
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------- distributed

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(val, ws):
    """Max over ranks (identity for one process)."""
    if ws == 1:
        return val
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(val)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------- CPU oracle leg

def cpu_sample(x_dev, w, frac_slices):
    """A bounded sample of the same tensor for the CPU oracle: the first time
    step and the first `frac_slices` slices of mode 2 (every other index
    kept), copied to the host in FP64."""
    import torch
    dims = w["dims"]
    rev = tuple(reversed(dims))
    t = x_dev.view(rev)
    idx = [slice(None)] * len(dims)
    # natural-descending mode n is torch dim N-1-n
    N = len(dims)
    if N >= 5:
        idx[N - 1 - 4] = slice(0, 1)
    if N >= 3:
        idx[N - 1 - 2] = slice(0, frac_slices)
    sub = t[tuple(idx)].contiguous()
    sdims = tuple(reversed(sub.shape))
    return sub.reshape(-1).double().cpu().numpy(), sdims


def run_cpu_oracle(xs, sdims, eps, recon_frac=None):
    """The oracle's step on the sample: ST-HOSVD, then the multi-TTM of a
    subtensor of the same relative size as the GPU step's (recon_frac: the
    fraction of the tensor the GPU step rebuilds, taken along mode 2 of the
    sample)."""
    import oracle
    t0 = time.perf_counter()
    res = oracle.sthosvd(xs, sdims, eps=eps)
    if recon_frac is not None:
        end = list(sdims)
        k = 2 if len(sdims) > 2 else 0
        end[k] = max(1, int(round(sdims[k] * recon_frac)))
        oracle.reconstruct(res["core"], res["core_dims"], res["factors"], (0,) * len(sdims), tuple(end))
    return time.perf_counter() - t0, res


def recon_frac(w):
    return float(np.prod(w["recon"])) / float(np.prod(w["dims"]))


def step(ctx, x, w, prec):
    """One pass of the hot path: ST-HOSVD (Algorithm 1) and the multi-TTM
    reconstruction (Section 7) of the workload's subtensor; returns the
    result (the reconstructed subtensor stays on the device)."""
    r = ctx.sthosvd(x, w["dims"], eps=w["eps"], prec=prec)
    rec = r.reconstruct((0,) * len(w["dims"]), w["recon"], prec=prec)
    del rec
    return r


def blas_threads():
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return len(os.sched_getaffinity(0))


# ---------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="large")
    ap.add_argument("--prec", choices=["mixed", "fp32", "fp64", "tensor"], default=None)
    ap.add_argument("--no-fp64", action="store_true", help="skip the one-step FP64-path leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-slices", type=int, default=None)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--autotune", type=int, default=1,
                    help="split-K autotuner of the Gram kernels (tuned during the warm-up)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)

    from paper_1901_06043_gb300 import synth, tucker

    w = WORKLOADS[args.workload]
    if "batch" in w:
        return main_batch(args, w, ws, rank)
    prec = args.prec or ("mixed" if tucker_mixed_available() else "fp32")
    if w["dtype"] == "f64" and prec == "mixed":
        prec = "fp32"
    tdt = torch.float32 if w["dtype"] == "f32" else torch.float64
    x = synth.tucker_torch(w["dims"], w["core"], decay=w["decay"], eta=w["eta"],
                           seed=args.seed + rank, dtype=tdt)
    torch.cuda.synchronize()
    in_bytes = x.numel() * x.element_size()
    N = len(w["dims"])
    cpu_slices = args.cpu_slices or (500 if args.workload == "large" else None)

    if args.impl == "reference":
        if rank != 0:
            return
        ref_ms = []
        xs, sdims = cpu_sample(x, w, cpu_slices or (w["dims"][2] if N >= 3 else None))
        del x
        for _ in range(args.warmup):
            run_cpu_oracle(xs, sdims, w["eps"], recon_frac(w))
        for _ in range(args.steps):
            t, _ = run_cpu_oracle(xs, sdims, w["eps"], recon_frac(w))
            ref_ms.append(t * 1e3)
        ms = statistics.mean(ref_ms)
        sbytes = xs.size * (4 if w["dtype"] == "f32" else 8)
        val = sbytes / 1e9 / (ms / 1e3)
        sample = f"oracle ST-HOSVD of the {'x'.join(map(str, sdims))} sub-tensor of the workload"
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {describe(w)}", "prec": "fp64-cpu-oracle"},
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": len(os.sched_getaffinity(0)),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return

    # warm-up on a context that records per-step CUDA events (kernel times for
    # the roofline); the timed steps below run on a context without them.  The
    # autotuner's cache is per process: the warm-up tunes, the timed steps reuse
    ctx_t = tucker.Context(timing=True)
    ctx = tucker.Context()
    for cx in (ctx_t, ctx):
        cx.set_option(tucker.OPT_AUTOTUNE, args.autotune)
    last = None
    for _ in range(args.warmup):
        if last is not None:
            last.close()
        last = ctx_t.sthosvd(x, w["dims"], eps=w["eps"], prec=prec)
    ranks = last.ranks
    ms_detail = dict(last.ms)
    # the reconstruction's own time (CUDA events on the library's stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    rec = last.reconstruct((0,) * len(w["dims"]), w["recon"], prec=prec)
    e1.record()
    torch.cuda.synchronize()
    ms_detail["recon"] = e0.elapsed_time(e1)
    rec_bytes = rec.numel() * rec.element_size()
    del rec
    pk = peaks()
    dom, step_rows = dominant(last, w, pk)
    last.close()
    torch.cuda.synchronize()
    # timed region
    clocks = Clocks(torch.cuda.current_device())
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    l0 = tucker.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        r = step(ctx, x, w, prec)
        r.close()
    ev1.record()
    torch.cuda.synchronize()
    launches = (tucker.kernel_launches() - l0) // args.steps
    barrier(ws)
    clk = clocks.stop()
    ms_local = ev0.elapsed_time(ev1) / args.steps
    ms = reduce_max(ms_local, ws)
    value = ws * in_bytes / 1e9 / (ms / 1e3)

    out = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec != "fp64" else "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {describe(w)}", "prec": prec,
                   "l2": "input larger than L2 (no flush)", "ranks": list(ranks),
                   "autotune": args.autotune,
                   "parallelism": f"replicas x{ws}"},
        "roofline": dom,
        "step": "ST-HOSVD (norm, Gram, eigensolve, rank cut, TTM per mode) + multi-TTM "
                f"reconstruction of the [0, {'x'.join(map(str, w['recon']))}) subtensor",
        "gpu_launches": int(launches),
        "clocks": clk,
        "per_mode_ms": {k: v for k, v in ms_detail.items()},
        "steps_roofline": [{k: r[k] for k in ("kernel", "ms", "bound", "achieved", "unit", "frac")
                            if k in r} for r in step_rows] +
                          [recon_roofline(ranks, w, ms_detail["recon"], rec_bytes, prec, pk)],
    }

    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_leg(ctx, x, w, prec, args)
    if rank == 0 and not args.no_fp64 and prec != "fp64":
        ctx_t.set_option(tucker.OPT_AUTOTUNE, 0)      # one untuned FP64 step
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        r64 = step(ctx_t, x, w, "fp64")
        t1.record()
        torch.cuda.synchronize()
        ms64 = t0.elapsed_time(t1)
        out["fp64_path"] = {"value": in_bytes / 1e9 / (ms64 / 1e3), "unit": "GB/s", "ms": ms64,
                            "steps": 1, "ranks": list(r64.ranks),
                            "ranks_equal": tuple(r64.ranks) == tuple(ranks),
                            "speedup_of_value": ms64 / ms_local, "per_mode_ms": r64.ms}
        r64.close()
    if rank == 0 and not args.no_cpu:
        xs, sdims = cpu_sample(x, w, cpu_slices if N >= 3 else None)
        t, _ = run_cpu_oracle(xs, sdims, w["eps"], recon_frac(w))
        sbytes = xs.size * (4 if w["dtype"] == "f32" else 8)
        out["cpu_baseline"] = {
            "value": sbytes / 1e9 / t, "unit": "GB/s", "cores": len(os.sched_getaffinity(0)),
            "blas_threads": blas_threads(), "kind": "oracle",
            "sample": (f"FP64 numpy oracle ST-HOSVD (Algorithm 1-3, eps {w['eps']:g}) of the "
                       f"{'x'.join(map(str, sdims))} sub-tensor of the workload "
                       f"({sbytes / 1e9:.2f} GB as {w['dtype']}) and the multi-TTM of "
                       f"{recon_frac(w):.3g} of it, {t:.1f} s")}
    if rank == 0:
        print(json.dumps(out))
    ctx.close()
    ctx_t.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main_batch(args, w, ws, rank):
    """The batched workload: one step = one tucker_sthosvd_batched call over
    all tensors (Algorithm 1 for each, lock-step by mode)."""
    import torch
    from paper_1901_06043_gb300 import synth, tucker
    prec = args.prec or ("mixed" if tucker_mixed_available() else "fp32")
    shapes = batch_shapes(w, args.seed + rank)
    xs = [synth.tucker_torch(d, c, decay=w["decay"], eta=w["eta"], seed=args.seed + rank + 7 * k)
          for k, (d, c) in enumerate(shapes)]
    dims_list = [d for d, _ in shapes]
    torch.cuda.synchronize()
    in_bytes = sum(t.numel() * t.element_size() for t in xs)
    if args.impl == "reference":
        if rank != 0:
            return
        # a bounded sample: the first tensors of the batch, on the host
        k = max(1, min(len(xs), args.cpu_slices or 8))
        hx = [t.double().cpu().numpy() for t in xs[:k]]
        del xs
        import oracle
        ref_ms = []
        for it in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            for xh, d in zip(hx, dims_list[:k]):
                oracle.sthosvd(xh, d, eps=w["eps"])
            if it >= args.warmup:
                ref_ms.append((time.perf_counter() - t0) * 1e3)
        ms = statistics.mean(ref_ms)
        sbytes = sum(a.size * 4 for a in hx)
        val = sbytes / 1e9 / (ms / 1e3)
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {describe(w)}", "prec": "fp64-cpu-oracle"},
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": len(os.sched_getaffinity(0)),
                             "kind": "oracle",
                             "sample": f"oracle ST-HOSVD of the first {k} tensors of the batch"},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return
    ctx = tucker.Context()
    ctx.set_option(tucker.OPT_AUTOTUNE, args.autotune)
    ranks = None
    for _ in range(args.warmup):
        rs = ctx.sthosvd_batched(xs, dims_list, w["eps"], prec=prec)
        ranks = [r.ranks for r in rs]
        for r in rs:
            r.close()
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    l0 = tucker.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        rs = ctx.sthosvd_batched(xs, dims_list, w["eps"], prec=prec)
        for r in rs:
            r.close()
    ev1.record()
    torch.cuda.synchronize()
    launches = (tucker.kernel_launches() - l0) // args.steps
    barrier(ws)
    clk = clocks.stop()
    ms_local = ev0.elapsed_time(ev1) / args.steps
    ms = reduce_max(ms_local, ws)
    value = ws * in_bytes / 1e9 / (ms / 1e3)
    pk = peaks()
    out = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec != "fp64" else "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {describe(w)}", "prec": prec,
                   "total_bytes": in_bytes, "l2": "inputs larger than L2 (no flush)",
                   "autotune": args.autotune,
                   "parallelism": f"replicas x{ws}"},
        # the whole step against HBM: every input byte is read at least once
        "roofline": {"bound": "hbm", "achieved": value, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": value / pk["hbm_gbs"], "traffic": None,
                     "kernel": "whole batched step (input bytes / step time)"},
        "step": "tucker_sthosvd_batched over all tensors",
        "gpu_launches": int(launches), "clocks": clk,
        "ranks_first": [list(r) for r in ranks[:4]],
    }
    if rank == 0 and not args.no_e2e:
        # host-resident inputs: pinned copies in, every core and factor out
        hx = [t.cpu().pin_memory() for t in xs]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps = max(1, args.steps)
        d2h = 0
        e0.record()
        for _ in range(steps):
            dx = [h.to("cuda", non_blocking=True) for h in hx]
            rs = ctx.sthosvd_batched(dx, dims_list, w["eps"], prec=prec)
            d2h = 0
            for r in rs:
                core, fac = r.to_host()
                d2h += core.nbytes + sum(f.nbytes for f in fac)
                r.close()
            del dx
        e1.record()
        torch.cuda.synchronize()
        ems = e0.elapsed_time(e1) / steps
        out["e2e"] = {"value": in_bytes / 1e9 / (ems / 1e3), "unit": "GB/s",
                      "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": d2h}
    print(json.dumps(out)) if rank == 0 else None
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def tucker_mixed_available():
    from paper_1901_06043_gb300 import tucker
    return getattr(tucker, "MIXED_AVAILABLE", False)


FP64_PEAK_TFLOPS = 1.19   # measured FP64 FMA throughput on this part (in-register probe)


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one ncu
# capture per kernel, with the input elements (I x K) that launch processed;
# a launch of the same kernel streams its input once, so its traffic scales
# with I x K.  Only kernels whose source has not changed since the capture.
# Both captures: `ncu --set full --clock-control none -k regex:<kernel> -c 1`
# of `bench.py --workload prof --steps 1 --warmup 3 --no-fp64 --no-e2e
# --no-cpu` (the 500x500x40x11x2 FP32 tensor), mode 0.
CAPTURED_TRAFFIC = {
    # k_gram_tcx (column mode, three digits), mode-0 Gram of 500x500x40x11x2
    # FP32: 741.3 GB/s x 1.192 ms
    ("gram", "tcgen05-x3", "col"): dict(bytes=883.3e6, elems=500 * 440000),
    # (no capture of the two-digit variant yet)
    # k_ttm_tc_col<64> (transposed output), mode-0 TTM of 500x500x40x11x2 FP32 to 54
    # rows: 4.553 TB/s x 212.2 us
    ("ttm", "tcgen05", "col"): dict(bytes=966.8e6, elems=500 * 440000),
}


def algorithmic_roofline(flops, nbytes, t, pk):
    """The roofline of a step from the work the method must do: the floor
    time is max(bytes / HBM copy bandwidth, flops / dense BF16 tensor peak),
    both measured on this part; frac = floor / measured time, `bound` the
    resource of the larger term, `achieved` that resource's rate."""
    t_hbm = nbytes / (pk["hbm_gbs"] * 1e9)
    t_flop = flops / (pk["bf16_tflops"] * 1e12)
    if t_hbm >= t_flop:
        return "hbm", nbytes / t / 1e9, pk["hbm_gbs"], "GB/s", t_hbm / t
    return "tensor", flops / t / 1e12, pk["bf16_tflops"], "TFLOP/s", t_flop / t


def step_rooflines(res, w, pk):
    """Roofline of every Gram / TTM / eigensolve step of one ST-HOSVD, from
    the library's own CUDA events on its stream.  Gram and TTM rows are
    rated on their algorithmic work (Gram I(I+1)K flops on I*K read
    elements; TTM 2RIK flops on I*K read + R*K written) against the HBM and
    tensor-core peaks, whichever binds; the eigensolves on their FP64 flops
    ((4/3) I^3 for the tridiagonal reduction, ~6 I^3 per Jacobi sweep)
    against the FP64 peak.  The digit Gram also reports its executed
    FP16 digit products against the tensor peak (mma_frac)."""
    ms, ranks = res.ms, res.ranks
    cur = list(w["dims"])
    # the natural mode order keeps the working tensor rotated: every mode's
    # Gram and TTM run on a column-mode view
    rotated = list(res.mode_order) == list(range(len(cur)))
    in_esz = 4 if w["dtype"] == "f32" else 8
    wk_esz = 8 if res.core_dtype == 1 else 4
    out = []
    for s, n in enumerate(res.mode_order):
        L = int(np.prod(cur[:n])) if n else 1
        I, R = cur[n], ranks[n]
        Rt = int(np.prod(cur[n + 1:])) if n + 1 < len(cur) else 1
        K = L * Rt
        esz = in_esz if s == 0 else wk_esz
        eig_k = "fp64-" + res.eig_kernel[n]
        eig_flops = (4.0 / 3.0) * I ** 3 if res.eig_kernel[n] == "tridiag" else \
            6.0 * I ** 3 * max(res.sweeps[n], 1)
        for kind, t_ms, flops, nbytes, kern in [
            ("gram", ms["gram"][n], I * (I + 1) * K, I * K * esz, res.gram_kernel[n]),
            ("ttm", ms["ttm"][n], 2 * R * I * K, I * K * esz + R * K * wk_esz, res.ttm_kernel[n]),
            ("eig", ms["eig"][n], eig_flops, 0, eig_k)]:
            t = max(t_ms, 1e-6) / 1e3
            traffic = None
            cap = CAPTURED_TRAFFIC.get((kind, kern, "col" if (L == 1 or rotated) else "row"))
            if cap is not None and I >= 64:
                traffic = cap["bytes"] * (I * K) / cap["elems"]
            extra = {}
            if kind == "eig":
                bound, ach, peak, unit = "alu", flops / t / 1e12, FP64_PEAK_TFLOPS, "TFLOP/s"
                frac = ach / peak
                src = "measured FP64 FMA probe"
            else:
                bound, ach, peak, unit, frac = algorithmic_roofline(flops, nbytes, t, pk)
                src = "measured HBM copy" if bound == "hbm" else "measured dense BF16 burst"
            if kern in ("tcgen05-x3", "tcgen05-x2"):
                # executed: 9 (three digits) or 4 (two) FP16 digit products per
                # product, on 128 x 128 lower-triangle tiles
                T = (I + 127) // 128
                nprod = 9 if kern == "tcgen05-x3" else 4
                mma = nprod * 2 * 128 * 128 * K * (T * (T + 1) // 2)
                extra = {"mma_tflops": mma / t / 1e12, "mma_frac": mma / t / 1e12 / pk["bf16_tflops"]}
            row = {"kernel": f"{kind} mode {n} ({kern})", "bound": bound, "achieved": ach,
                   "peak": peak, "unit": unit, "frac": frac, "traffic": traffic,
                   "ms": t_ms, "algorithmic_bytes": nbytes, "algorithmic_flops": flops,
                   "peak_src": src}
            row.update(extra)
            if traffic is not None:
                row["traffic_src"] = ("ncu DRAM bytes of the same kernel on the 500x500x40x11x2 "
                                      "FP32 tensor, scaled by I*K")
            out.append(row)
        cur[n] = R
    return out


def recon_roofline(ranks, w, ms, out_bytes, prec, pk):
    """The multi-TTM reconstruction of the step: its algorithmic work is the
    subtensor it writes (out_bytes) and the flops of the chain order the
    library picks (sum over the chain of 2 x output elements x contracted
    rank); rated like the Gram and TTM rows (HBM or tensor peak, whichever
    binds)."""
    from paper_1901_06043_gb300 import tucker
    order = tucker.ttm_order(ranks, w["recon"], "flops")
    cur = list(ranks)
    flops = 0.0
    for n in order:
        cur[n] = w["recon"][n]
        flops += 2.0 * float(np.prod(cur)) * ranks[n]
    t = ms / 1e3
    bound, ach, peak, unit, frac = algorithmic_roofline(flops, out_bytes, t, pk)
    return {"kernel": f"multi-TTM reconstruction (order {list(order)})", "ms": ms, "bound": bound,
            "achieved": ach, "peak": peak, "unit": unit, "frac": frac,
            "algorithmic_bytes": out_bytes, "algorithmic_flops": flops}


def dominant(res, w, pk):
    """The longest step's roofline entry."""
    rows = step_rooflines(res, w, pk)
    return max(rows, key=lambda r: r["ms"]), rows


class HostBuffer:
    """A page-locked host buffer of n elements: anonymous memory mapped by
    this process (huge pages where the kernel allows), every page touched by
    the CPU, then registered with CUDA (cudaHostRegister).  After a process
    has churned through the host's memory, buffers from the CUDA host
    allocator measured up to 3x slower device-to-host copies on this machine
    (~66 against ~193 GB/s); buffers made this way kept the full rate."""

    def __init__(self, n, dtype):
        import ctypes
        import mmap
        import torch
        esize = torch.empty(0, dtype=dtype).element_size()
        nbytes = max(1, n * esize)
        self._m = mmap.mmap(-1, nbytes, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        self._addr = ctypes.addressof(ctypes.c_char.from_buffer(self._m))
        try:
            libc = ctypes.CDLL("libc.so.6")
            libc.madvise.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
            libc.madvise(self._addr, nbytes, 14)          # MADV_HUGEPAGE; advisory
        except OSError:
            pass
        raw = np.frombuffer(self._m, dtype=np.uint8)
        raw[::4096] = 0                                    # fault every page in
        st = torch.cuda.cudart().cudaHostRegister(self._addr, nbytes, 0)
        self.registered = int(st) == 0
        npdt = {torch.float32: np.float32, torch.float64: np.float64}[dtype]
        self.tensor = torch.from_numpy(np.frombuffer(self._m, dtype=npdt, count=n))

    def close(self):
        import torch
        self.tensor = None
        if self.registered:
            torch.cuda.cudart().cudaHostUnregister(self._addr)
            self.registered = False


def e2e_leg(ctx, x, w, prec, args):
    """Same metric end to end: the step through the C ABI from a pinned host
    input (tucker_sthosvd_host: the library copies the tensor in pieces and
    runs the norm pass and the mode-0 Gram on each piece as it lands), the
    subtensor reconstruction, and the reconstructed subtensor, the core and
    the factors back to pinned host memory, per step.  `value` is the rate of
    two host threads running such steps at once (e2e_streams); `serial` is
    that of one thread."""
    import torch
    xb = HostBuffer(x.numel(), x.dtype)
    rb = HostBuffer(int(np.prod(w["recon"])), x.dtype)
    xh, rh = xb.tensor, rb.tensor
    pinned = xb.registered and rb.registered
    xh.copy_(x)
    steps = max(1, min(args.steps, 3))
    # the plain host-to-device rate of every 4 GB piece of this pinned
    # buffer, for reading the figure: the copy bounds the end-to-end step, and
    # on this machine some pieces of a fresh buffer copied at a tenth of the
    # rate after other processes had used the host's memory
    nprobe = min(xh.numel(), (4 << 30) // xh.element_size())
    scratch = torch.empty(nprobe, dtype=xh.dtype, device="cuda")
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    slice_gbs = []
    for k in range(0, xh.numel(), nprobe):
        m = min(nprobe, xh.numel() - k)
        h0.record()
        scratch[:m].copy_(xh[k:k + m], non_blocking=True)
        h1.record()
        torch.cuda.synchronize()
        slice_gbs.append(round(m * xh.element_size() / 1e6 / h0.elapsed_time(h1), 1))
    h2d_gbs = float(np.median(slice_gbs))
    del scratch
    # one untimed call: the autotuner's first visit of the piece shapes
    ctx.sthosvd_host(xh, w["dims"], eps=w["eps"], prec=prec).close()
    torch.cuda.synchronize()
    d2h = 0
    t0 = time.perf_counter()
    step_ms = []
    for _ in range(steps):
        ts = time.perf_counter()
        r = ctx.sthosvd_host(xh, w["dims"], eps=w["eps"], prec=prec)
        rec = r.reconstruct((0,) * len(w["dims"]), w["recon"], prec=prec)
        rh.copy_(rec.view(-1).to(rh.dtype), non_blocking=True)
        core, fac = r.to_host()
        torch.cuda.synchronize()
        d2h = rh.numel() * rh.element_size() + core.nbytes + sum(f.nbytes for f in fac)
        del rec
        r.close()
        step_ms.append((time.perf_counter() - ts) * 1e3)
    torch.cuda.synchronize()
    el = (time.perf_counter() - t0) / steps
    nb = x.numel() * x.element_size()
    serial = {"value": nb / 1e9 / el, "ms": el * 1e3, "steps": steps, "step_ms": step_ms}
    del rh
    rb.close()
    par = e2e_streams(xh, w, prec, args, nstreams=2, per_stream=3)
    del xh
    xb.close()
    el = par["ms"] / 1e3
    return {"value": nb / 1e9 / el, "unit": "GB/s", "h2d_bytes_per_step": nb,
            "d2h_bytes_per_step": int(d2h), "steps": par["steps"], "streams": par["streams"],
            "pinned": pinned, "ms": par["ms"], "wall_ms": par["wall_ms"],
            "h2d_copy_gbs": h2d_gbs, "h2d_copy_gbs_per_4gb": slice_gbs,
            "returns": "reconstructed subtensor, core and factors",
            "serial": serial}


def e2e_streams(xh, w, prec, args, nstreams=2, per_stream=2):
    """The end-to-end steps from `nstreams` host threads, each with its own
    context on its own CUDA stream and its own pinned output buffer, all
    reading the same pinned input: while one thread's step computes and
    copies its results back, another's input copy is under way, so the
    host-to-device link stays busy.  Every step still copies its whole input
    in and its reconstructed subtensor, core and factors out.  Results stay
    open until the timed region ends (closing one synchronizes the device).
    Returns the wall time per step over all threads' steps."""
    import threading
    import torch
    from paper_1901_06043_gb300 import tucker
    streams = [torch.cuda.Stream() for _ in range(nstreams)]
    ctxs, outs = [], []
    for s in streams:
        with torch.cuda.stream(s):
            c = tucker.Context(stream=s.cuda_stream)
        c.set_option(tucker.OPT_AUTOTUNE, args.autotune)
        ctxs.append(c)
        outs.append(HostBuffer(int(np.prod(w["recon"])), xh.dtype))
    keep = [[] for _ in range(nstreams)]
    errors = []

    def run(i, n):
        try:
            with torch.cuda.stream(streams[i]):
                for _ in range(n):
                    r = ctxs[i].sthosvd_host(xh, w["dims"], eps=w["eps"], prec=prec)
                    rec = r.reconstruct((0,) * len(w["dims"]), w["recon"], prec=prec)
                    outs[i].tensor.copy_(rec.view(-1).to(outs[i].tensor.dtype), non_blocking=True)
                    r.to_host()
                    streams[i].synchronize()
                    del rec
                    keep[i].append(r)
        except Exception as e:                 # re-raised after the join
            errors.append(e)

    def close_all():
        for lst in keep:
            for r in lst:
                r.close()
            lst.clear()

    def run_all(n):
        threads = [threading.Thread(target=run, args=(i, n)) for i in range(nstreams)]
        t0 = time.perf_counter()
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if errors:
            raise errors[0]
        return time.perf_counter() - t0

    # untimed: one call per context, all at once, so that the memory pool
    # holds every context's working set before the timed steps
    run_all(1)
    close_all()
    torch.cuda.synchronize()
    wall = run_all(per_stream)
    close_all()
    for c in ctxs:
        c.close()
    for o in outs:
        o.close()
    steps = nstreams * per_stream
    return {"ms": wall * 1e3 / steps, "wall_ms": wall * 1e3, "steps": steps, "streams": nstreams}


if __name__ == "__main__":
    main()
