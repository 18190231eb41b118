#!/usr/bin/env python3
"""Benchmark: staged 3D FFT at 512^3 FP32 on GB300 (one JSON line on stdout).

Workload (the real-data full-size configuration): R2C forward then C2R
inverse of a 512x512x512 float32 grid, real N(0,1) input (seed 2), pencil
stages x -> y -> z in one persistent launch per transform. One step = one
forward + one inverse. Inputs (512 MiB real, 539 MB spectrum) are larger than
the 129 MB L2, so no flush is needed between steps.

  value      GFLOP/s, 5 N log2 N per transform (the metric's convention; for a
             real transform this is twice the 2.5 N log2 N real-flop count,
             also reported), whole job over all ranks
  e2e        the same metric through gbfft_exec_host on pinned HOST buffers
             (H2D + exec + D2H inside the timed region)
  roofline   the persistent kernel: algorithmic HBM bytes per launch / CUDA-event
             launch time, against the measured copy bandwidth
  cpu_baseline  the FP64 oracle on the host cores (one full step)

--impl reference times the FP64 CPU oracle itself (the only reference this
project has) on a bounded sample of the same workload.
Multi-GPU (torchrun): independent replicas, one per GPU ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 512
METRIC = "3D FFT GFLOP/s (5N*log2N) at 512^3 FP32, R2C fwd + C2R inv per step"
UNIT = "GFLOP/s"


def flops_5n(nx, ny, nz):
    n = nx * ny * nz
    return 5.0 * n * math.log2(n)


def r2c_alg_bytes(nx, ny, nz):
    """Algorithmic HBM bytes of one pencil R2C (or C2R) transform: the real
    array once (4 B/elem), the half spectrum written by x, read+written by y
    and z, read... i.e. 3 reads + 3 writes of the stage arrays."""
    nc = (nx // 2 + 1) * ny * nz
    return 4 * nx * ny * nz + 5 * 8 * nc


def c2c_alg_bytes(nx, ny, nz, passes=3):
    return passes * 2 * 8 * nx * ny * nz


def slab_r2c_alg_bytes(nx, ny, nz):
    nc = (nx // 2 + 1) * ny * nz
    return 4 * nx * ny * nz + 3 * 8 * nc


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# the sources of the stage, tensor-copy and warp-per-pencil kernels' device code
KERNEL_SOURCES = ("gbfft_internal.h", "gbfft_device.cuh", "gbfft_kernels.cuh", "gbfft_tma.cuh", "gbfft_warp.cuh",
                  "gbfft_warp_tile.cuh", "gbfft_prefetch.cuh")
# ... and of the fused plane kernels
PLANE_SOURCES = KERNEL_SOURCES + ("gbfft_plane.cuh",)


def kernel_source_hash(files=KERNEL_SOURCES):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2601_12209_gb300", "csrc")
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key):
    """Per-launch DRAM bytes from the committed ncu summary, if taken on the current kernels."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic_r2c_512.json")
    if not os.path.exists(p):
        return None
    try:
        with open(p) as fh:
            d = json.load(fh)
        if "plane" in kernel_key:
            if d.get("plane_source_hash") != kernel_source_hash(PLANE_SOURCES):
                return None
        elif d.get("source_hash") != kernel_source_hash():
            return None
        v = d.get("kernels", {}).get(kernel_key)
        return float(v) if v is not None else None
    except Exception:
        return None


def _parse_cpulist(text):
    cpus = set()
    for part in text.strip().split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    return cpus


def bind_near_gpu(torch, device_index):
    """Run this process on the CPUs of the NUMA node the GPU is attached to (from sysfs), so that
    pinned host buffers allocated afterwards sit next to the GPU's link. Returns the node or None."""
    try:
        uuid = str(torch.cuda.get_device_properties(device_index).uuid)
        ident = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        bus = subprocess.run(["nvidia-smi", f"--id={ident}", "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        dom, rest = bus.split(":", 1)
        with open(f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest.lower()}/numa_node") as fh:
            node = int(fh.read().strip())
        if node < 0:
            return None
        with open(f"/sys/devices/system/node/node{node}/cpulist") as fh:
            local = _parse_cpulist(fh.read()) & os.sched_getaffinity(0)
        if local:
            os.sched_setaffinity(0, local)
        return node
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max_ms(dist, ms: float, device) -> float:
    """Max of a per-rank time over all ranks (the slowest replica sets the job time)."""
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, flops_per_step: float, ms_per_step: float) -> float:
    """GFLOP/s of the whole job: every replica does one step's work per ms_per_step."""
    return world * flops_per_step / (ms_per_step * 1e-3) / 1e9


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The FP64 oracle on the host cores, on the same workload as the GPU arm: each step is the
    R2C forward + C2R inverse of the 512^3 grid (seed 2), about 3 s per step on 16 cores."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import numpy as np
    import oracle
    import synth
    n = N
    r = synth.normal_real((n, n, n), seed=2).numpy().astype(np.float64)
    threads = oracle.default_threads()
    for _ in range(args.warmup):
        oracle.irfft3(oracle.rfft3(r, threads=threads), n, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.irfft3(oracle.rfft3(r, threads=threads), n, threads=threads)
    dt = (time.perf_counter() - t0) / args.steps
    value = 2 * flops_5n(n, n, n) / dt / 1e9
    sample = f"R2C fwd + C2R inv of the 512^3 grid in FP64 per step (the full workload), {threads} threads"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "R2C fwd + C2R inv 3D FFT 512x512x512 FP32, pencil stages x-y-z, autotuned launches",
                   "nx": n, "ny": n, "nz": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_oracle(spec_gpu=None, real_gpu=None):
    """One full 512^3 R2C fwd + C2R inv step of the FP64 oracle on all host cores. From the same
    oracle outputs it also checks the timed loop's own results (the last step's spectrum and
    real output, copied from the device): rel-L2 of the forward and of the round trip."""
    import numpy as np
    import oracle
    import synth
    r = synth.normal_real((N, N, N), seed=2).numpy().astype(np.float64)
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    ref = oracle.rfft3(r, threads=threads)
    oracle.irfft3(ref, N, threads=threads)
    dt = time.perf_counter() - t0
    base = {"value": 2 * flops_5n(N, N, N) / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"one full step (512^3 R2C fwd + C2R inv, FP64) in {dt:.2f} s"}
    parity = None
    if spec_gpu is not None and real_gpu is not None:
        parity = {"rel_l2_fwd": oracle.rel_l2(spec_gpu.reshape(ref.shape), ref),
                  "rel_l2_roundtrip": oracle.rel_l2(real_gpu.reshape(r.shape), r),
                  "tol": 1e-5, "against": "FP64 oracle on the same seed-2 input; outputs of the last timed step"}
        parity["ok"] = parity["rel_l2_fwd"] <= 1e-5 and parity["rel_l2_roundtrip"] <= 1e-5
    return base, parity


def time_variant(torch, plan, x, ops, steps, warmup, stream):
    """Per-launch CUDA-event times of a list of (op, input-from) exec calls per step."""
    bufs = {"x": x}
    for _ in range(warmup):
        cur = x
        for op in ops:
            cur = plan.exec(op, cur, stream=stream)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(ops) + 1)] for _ in range(steps)]
    with torch.cuda.stream(stream):
        for s in range(steps):
            cur = x
            ev[s][0].record(stream)
            for i, op in enumerate(ops):
                cur = plan.exec(op, cur, stream=stream)
                ev[s][i + 1].record(stream)
    torch.cuda.synchronize()
    per = [[ev[s][i].elapsed_time(ev[s][i + 1]) for s in range(steps)] for i in range(len(ops))]
    del bufs
    return [statistics.median(p) for p in per], [sum(p) / len(p) for p in per]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gbfft", choices=["gbfft", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--launch", default="auto", choices=["auto", "persistent", "staged"],
                    help="auto: autotune the plan; persistent / staged: fix the launch choice")
    ap.add_argument("--tma-mask-fwd", type=int, default=0, help="with --launch staged: tensor-copy stages (bits)")
    ap.add_argument("--tma-mask-inv", type=int, default=0, help="with --launch staged: tensor-copy stages (bits)")
    ap.add_argument("--ncu-case", default=None,
                    help="run one 512^3 case for a profiler and exit: staged_r2c, staged_lsu_r2c, persistent_r2c, "
                         "staged_c2c, staged_lsu_c2c, persistent_c2c, slab_c2c, slab_r2c; or split_fp16_1024, "
                         "split_bf16_1024, split_fp16_tc5_1024, split_bf16_tc5_1024, split_fp32_1024 (C2C "
                         "1024x512x64, staged thread-load launches; tensor-core radix-16 passes unless fp32); "
                         "or pinned_r2c:<fwd bits>:<inv bits> (pinned_slab_r2c: slab plan), dsm_slab_r2c (R2C 512x512x128 slab, "
                         "plane launches in distributed shared memory), batched_64 / batched_64_staged (the 64 uneven "
                         "grids, one launch / three stage launches), persistent_warp_c2c (C2C 512^3, one persistent "
                         "launch with warp-per-pencil tile bodies), warp1024_c2c (C2C 1024x512x64, warp-per-pencil "
                         "stages)")
    args = ap.parse_args()
    if args.ncu_case:
        ncu_case(args.ncu_case)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import synth
    world, rank, local = dist_setup(args)
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2601_12209_gb300 import _build
    if rank == 0 or world == 1:
        _build.build()
    if dist:
        dist.barrier()
    import paper_2601_12209_gb300 as gb
    from paper_2601_12209_gb300 import abi

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    plan = gb.Plan(N, N, N, kind="r2c")
    if args.launch == "auto":
        tuning = plan.autotune(stream)  # picks per-stage kernels or the persistent launch (outside the timed region)
    else:  # a fixed choice, e.g. to profile exactly what an earlier autotuned run chose
        for k, (pers, mask) in enumerate(((args.launch == "persistent", args.tma_mask_fwd),
                                          (args.launch == "persistent", args.tma_mask_inv))):
            abi.gbfft_plan_set_tuning(plan.handle, k, pers, mask)
        tuning = {name: abi.gbfft_plan_get_tuning(plan.handle, k) for k, name in enumerate(("forward", "inverse"))}
    r = synth.normal_real((N, N, N), seed=2).to(dev)
    spec = torch.empty((1, N, N, N // 2 + 1), dtype=torch.complex64, device=dev)
    real_out = torch.empty((1, N, N, N), dtype=torch.float32, device=dev)

    def step():
        plan.exec(abi.GBFFT_OP_FORWARD, r, spec, stream)
        plan.exec(abi.GBFFT_OP_INVERSE, spec, real_out, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    sampler = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
                           if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    abi.gbfft_plan_time_stages(plan.handle, True)
    sampler.start()
    time.sleep(0.3)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 1)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        t_start.record(stream)
        for s in range(args.steps):
            evs[2 * s].record(stream)
            plan.exec(abi.GBFFT_OP_FORWARD, r, spec, stream)
            evs[2 * s + 1].record(stream)
            plan.exec(abi.GBFFT_OP_INVERSE, spec, real_out, stream)
            evs[2 * s + 2].record(stream)
        t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    abi.gbfft_plan_time_stages(plan.handle, False)
    seg_fwd, _ = abi.gbfft_plan_stage_times(plan.handle, 0)
    seg_inv, _ = abi.gbfft_plan_stage_times(plan.handle, 1)
    total_ms = t_start.elapsed_time(t_end)
    fwd_ms = [evs[2 * s].elapsed_time(evs[2 * s + 1]) for s in range(args.steps)]
    inv_ms = [evs[2 * s + 1].elapsed_time(evs[2 * s + 2]) for s in range(args.steps)]
    if dist:
        total_ms = reduce_max_ms(dist, total_ms, dev)
    ms_per_step = total_ms / args.steps
    flops_step = 2 * flops_5n(N, N, N)
    value = whole_job_value(world, flops_step, ms_per_step)
    err = plan.device_error()

    # roofline of the dominant launch: per-launch CUDA events recorded by the
    # library on the launching stream during the timed loop
    peak, peak_kind = measured_peaks()
    nc = (N // 2 + 1) * N * N
    nreal = N * N * N
    segs = []
    for name, seg, tune, stage_bytes in (
            ("forward", seg_fwd, tuning["forward"], [4 * nreal + 8 * nc, 16 * nc, 16 * nc]),
            ("inverse", seg_inv, tuning["inverse"], [16 * nc, 16 * nc, 8 * nc + 4 * nreal])):
        if tune["persistent"] or len(seg) == 1:
            segs.append((f"{name} persistent_kernel", seg[0], sum(stage_bytes)))
        else:
            axes = ("x", "y", "z") if name == "forward" else ("z", "y", "x")
            for k, t in enumerate(seg):
                # the warp kernel serves the complex length-512 stages (y, z), not the real x stages
                kern = ("c2r_prefetch_kernel" if k < 4 and (tune["tma_mask"] >> (28 + k)) & 1 else
                        "warp_stage_kernel" if (tune["tma_mask"] >> (20 + k)) & 1 and axes[k] != "x" else
                        "tma_stage_kernel" if (tune["tma_mask"] >> k) & 1 else "stage_kernel")
                segs.append((f"{name} stage {axes[k]} {kern}", t, stage_bytes[k]))
    dom = max(segs, key=lambda x: x[1])
    bytes_launch = dom[2]
    avg_launch_ms = dom[1]
    achieved = bytes_launch / (avg_launch_ms * 1e-3) / 1e9
    traffic = ncu_traffic(dom[0])
    launches_per_step = sum(1 if t["persistent"] else 3 for t in (tuning["forward"], tuning["inverse"]))

    # end to end through the C ABI on pinned host buffers, allocated on the GPU's NUMA node
    numa_node = bind_near_gpu(torch, dev.index if dev.index is not None else 0)
    h_in = synth.normal_real((N, N, N), seed=2).pin_memory()
    h_spec = torch.empty((N, N, N // 2 + 1), dtype=torch.complex64).pin_memory()
    h_out = torch.empty((N, N, N), dtype=torch.float32).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))

    def e2e_round(chunks):
        plan.set_host_chunks(chunks)
        plan.exec_host(abi.GBFFT_OP_FORWARD, h_in, h_spec)
        plan.exec_host(abi.GBFFT_OP_INVERSE, h_spec, h_out)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            plan.exec_host(abi.GBFFT_OP_FORWARD, h_in, h_spec)
            plan.exec_host(abi.GBFFT_OP_INVERSE, h_spec, h_out)
        return (time.perf_counter() - t0) / e2e_steps

    # same process, same buffers: the one-copy path and the chunked path (copies overlapped with the first and
    # last stages), alternated over five rounds; the faster configuration is the reported e2e
    ab = {1: [], 8: []}
    for _ in range(5):
        for chunks in (1, 8):
            ab[chunks].append(e2e_round(chunks))
    e2e_chunks = min(ab, key=lambda c: statistics.median(ab[c]))
    e2e_s = statistics.median(ab[e2e_chunks])
    plan.set_host_chunks(1)
    e2e_val = world * flops_step / e2e_s / 1e9
    h2d = h_in.numel() * 4 + h_spec.numel() * 8
    d2h = h_spec.numel() * 8 + h_out.numel() * 4

    extra = {}
    if not args.no_extra and rank == 0:
        extra = extra_variants(torch, gb, abi, dev, stream, max(5, args.steps // 2), 3)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "R2C fwd + C2R inv 3D FFT 512x512x512 FP32, pencil stages x-y-z, autotuned launches",
                   "nx": N, "ny": N, "nz": N, "kind": "r2c", "decomposition": "pencil",
                   "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas" if world > 1 else "1gpu",
                   "flop_convention": "5 N log2 N per transform (real-flop count 2.5 N log2 N is half)"},
        "gflops_real_convention": value / 2,
        "fwd_ms": statistics.median(fwd_ms), "inv_ms": statistics.median(inv_ms),
        "hbm_gbs_algorithmic": 2 * r2c_alg_bytes(N, N, N) / (ms_per_step * 1e-3) / 1e9,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": dom[0], "bytes_per_launch": bytes_launch,
                     "avg_launch_ms": avg_launch_ms, "peak_source": f"{peak_kind} hbm_gbs",
                     "launches": [{"launch": n, "avg_ms": t, "alg_bytes": b, "gbs": b / (t * 1e-3) / 1e9}
                                  for (n, t, b) in segs]},
        "step_roofline_frac": 2 * r2c_alg_bytes(N, N, N) / (ms_per_step * 1e-3) / 1e9 / peak,
        "tuning": {k: {"persistent": v["persistent"], "tma_mask": v["tma_mask"], "ms": v["ms"]}
                   for k, v in tuning.items()},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_s * 1e3, "path": "gbfft_exec_host (pinned host buffers)",
                "host_chunks": e2e_chunks,
                "ab_ms_per_step": {f"chunks_{c}": [round(v * 1e3, 3) for v in ab[c]] for c in ab},
                "host_numa_node": numa_node},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "device_error": err,
        "extra": extra,
    }
    if rank == 0 and not args.no_cpu_baseline:
        del h_in, h_spec, h_out
        # the timed loop's own outputs (the last step's spectrum and real output)
        line["cpu_baseline"], line["parity"] = cpu_baseline_oracle(spec.cpu().numpy(), real_out.cpu().numpy())
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def ncu_case(name):
    """Three forward+inverse pairs of one 512^3 configuration, nothing timed (for ncu)."""
    import torch
    import synth
    import paper_2601_12209_gb300 as gb
    from paper_2601_12209_gb300 import _build, abi
    _build.build()
    if name.startswith("batched_64"):
        # batched_64 / batched_64_staged: the 64 uneven C2C grids (72.4 M points), tuned tile shapes, three forward
        # transforms as the one launch or as the three stage launches
        shapes, grids = synth.batched_grids(64, seed=6)
        m = gb.ManyPlan(shapes)
        x = m.pack([g.cuda() for g in grids])
        y = m.empty()
        # the autotuner's choice on this configuration (tiles per ticket by axis length), set by hand so that
        # the profiled launches follow few others
        m.set_tuning(0, {32: 4, 48: 4, 60: 2, 64: 2, 80: 2, 96: 2, 120: 2, 128: 2, 160: 1, 192: 1, 256: 1})
        torch.cuda.synchronize()
        run = m.exec_staged if name.endswith("staged") else m.exec
        for _ in range(3):
            run(abi.GBFFT_OP_FORWARD, x, y)
        torch.cuda.synchronize()
        return
    if name.startswith("split_"):
        # split_<fp16|bf16|fp32>[_tc5]_1024: C2C 1024 x 512 x 64 (268 MB per buffer), x stage has the tensor-core
        # pass (warp-level mma.sync, or tcgen05 with _tc5)
        parts = name.split("_")
        prec = parts[1]
        tc5 = "tc5" in parts
        plan = gb.Plan(1024, 512, 64, precision=prec if prec == "fp32" else prec + "_split" + ("_tc5" if tc5 else ""),
                       staged=True, tma=False)
        x = synth.uniform_complex((64, 512, 1024), seed=3).cuda()
        kind = "c2c"
    elif name == "persistent_warp_c2c":
        # C2C 512^3 as one persistent launch per transform, warp-per-pencil tile body on all three stages
        kind = "c2c"
        plan = gb.Plan(N, N, N)
        for k in (0, 1):
            abi.gbfft_plan_set_tuning(plan.handle, k, True, 0x7 << 20)
        x = synth.uniform_complex((N, N, N), seed=3).cuda()
    elif name == "warp1024_c2c":
        # C2C 1024 x 512 x 64 (268 MB per buffer): the x stage on the length-1024 warp-per-pencil kernel
        kind = "c2c"
        plan = gb.Plan(1024, 512, 64, staged=True)
        for k in (0, 1):
            abi.gbfft_plan_set_tuning(plan.handle, k, False, 0x1F << 20)
        x = synth.uniform_complex((64, 512, 1024), seed=3).cuda()
    elif name == "dsm_slab_r2c":
        # R2C 512 x 512 x 128 slab (128 MiB real in, 135 MB spectrum out): the in-plane pairs as plane launches
        # with the intermediate in distributed shared memory
        kind = "r2c"
        plan = gb.Plan(N, N, 128, kind=kind, slab=True)
        abi.gbfft_plan_set_tuning(plan.handle, 0, False, (1 << 27) | (1 << 8))
        abi.gbfft_plan_set_tuning(plan.handle, 1, False, (1 << 27) | (2 << 8))
        x = synth.normal_real((128, N, N), seed=2).cuda()
    elif name.startswith("pinned_r2c") or name.startswith("pinned_slab_r2c"):
        # pinned_r2c:<forward bits>:<inverse bits>: R2C 512^3 with a fixed launch choice (the tuning bits of
        # gbfft_plan_set_tuning), e.g. the benchmark's autotuned choice, so a profile sees the timed kernels;
        # pinned_slab_r2c: the same for a slab plan
        _, fwd, inv = name.split(":")
        kind = "r2c"
        plan = gb.Plan(N, N, N, kind=kind, slab=name.startswith("pinned_slab"))
        abi.gbfft_plan_set_tuning(plan.handle, 0, False, int(fwd, 0))
        abi.gbfft_plan_set_tuning(plan.handle, 1, False, int(inv, 0))
        x = synth.normal_real((N, N, N), seed=2).cuda()
    else:
        kind = "r2c" if name.endswith("r2c") else "c2c"
        plan = gb.Plan(N, N, N, kind=kind, staged=name.startswith("staged"), slab=name.startswith("slab"),
                       tma="_lsu" not in name)
        x = (synth.normal_real((N, N, N), seed=2) if kind == "r2c" else synth.uniform_complex((N, N, N), seed=3)).cuda()
    for _ in range(3):
        y = plan.exec(abi.GBFFT_OP_FORWARD, x)
        plan.exec(abi.GBFFT_OP_INVERSE, y)
    torch.cuda.synchronize()
    assert plan.device_error() == 0


def batched_variant(torch, gb, abi, stream, steps, warmup):
    """64 uneven C2C grids (forward): the graph-captured one launch with one 16-pencil tile per
    ticket, then the tile-shape autotuner's choice in all three schedules."""
    import synth
    shapes, grids = synth.batched_grids(64, seed=6)
    m = gb.ManyPlan(shapes)
    x = m.pack([g.cuda() for g in grids])
    y = m.empty()
    npts = sum(nx * ny * nz for (nx, ny, nz) in shapes)
    flops = sum(flops_5n(*s) for s in shapes)
    alg_bytes = 48 * npts
    res = {"grids": 64, "points": npts, "alg_bytes": alg_bytes,
           "largest_smallest_ratio": max(a * b * c for a, b, c in shapes) / min(a * b * c for a, b, c in shapes)}

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                fn()
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        return {"ms": ms, "gflops": flops / (ms * 1e-3) / 1e9, "alg_gbs": alg_bytes / (ms * 1e-3) / 1e9}

    def graph_of(fn):
        with torch.cuda.stream(stream):
            fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            fn()
        return g

    one = lambda: m.exec(abi.GBFFT_OP_FORWARD, x, y, stream=stream)  # noqa: E731
    g1 = graph_of(one)
    res["one_launch_graph_one_tile_per_ticket"] = timed(lambda: g1.replay())
    del g1
    res["tuning"] = {k: {"tiles_per_ticket": v["teams"], "queue_lag": v["lag"], "ms": v["ms"]}
                     for k, v in m.autotune(stream).items()}
    graph = graph_of(one)
    graph3 = graph_of(lambda: m.exec_staged(abi.GBFFT_OP_FORWARD, x, y, stream=stream))
    for name, fn in (("one_launch_graph", lambda: graph.replay()),
                     ("stage_launches_graph", lambda: graph3.replay()),
                     ("one_launch", one),
                     ("separate_plans", lambda: m.exec_separate(abi.GBFFT_OP_FORWARD, x, y, stream=stream))):
        res[name] = timed(fn)
    res["device_error"] = m.device_error()
    m.close()
    return res


def poisson_variant(torch, gb, abi, stream, steps, warmup):
    """Periodic Poisson solve on 256^3 (R2C, multiplier fused into the z stage, C2R)."""
    import synth
    n = 256
    f, _ = synth.poisson_rhs(n, seed=4)
    f = f.cuda()
    p = gb.Plan(n, n, n, kind="r2c")
    tune = p.autotune(stream)
    phi = torch.empty_like(f)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            p.poisson(f, phi, stream=stream)
        e0.record(stream)
        for _ in range(steps):
            p.poisson(f, phi, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    nc = (n // 2 + 1) * n * n
    alg = 2 * (4 * n ** 3 + 8 * nc) + 2 * 16 * nc + 16 * nc  # x, y out and back; fused z: one read + one write
    out = {"ms": ms, "alg_gbs": alg / (ms * 1e-3) / 1e9, "tuning": tune["poisson"]}
    # (Periodic, Periodic, Bounded): the same pipeline with the DCT z stage
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            p.poisson(f, phi, stream=stream, bounded=True)
        e0.record(stream)
        for _ in range(steps):
            p.poisson(f, phi, stream=stream, bounded=True)
        e1.record(stream)
    torch.cuda.synchronize()
    msb = e0.elapsed_time(e1) / steps
    out["bounded_z"] = {"ms": msb, "alg_gbs": alg / (msb * 1e-3) / 1e9}
    p.close()
    return out


def precision_variant(torch, gb, abi, stream, steps, warmup):
    """1024^3 C2C: FP32 butterflies vs tensor-core radix-16 passes with FP16 / BF16 hi/lo pairs, as
    warp-level mma.sync products and as tcgen05.mma products with tensor-memory accumulators.

    Timing input: uniform[-1,1] noise drawn on the device from a seeded generator plus 16
    plane waves (the FFT's work does not depend on the values). Accuracy without the oracle:
    the waves alone against their closed form n^3 a_m (peak error, energy leaked elsewhere)
    and the round trip of the full input.
    """
    import numpy as np
    import synth
    n = 1024
    N = n ** 3
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    x = torch.complex(torch.rand((n, n, n), generator=g, device="cuda") * 2 - 1,
                      torch.rand((n, n, n), generator=g, device="cuda") * 2 - 1)
    ks, amps = synth.plane_wave_spec(n, seed=7)
    synth.add_plane_waves(x, ks, amps)
    waves = synth.add_plane_waves(torch.zeros_like(x), ks, amps)
    pk = torch.as_tensor(ks, device="cuda")
    out = {"grid": [n, n, n], "flops_5nlog2n": flops_5n(n, n, n), "alg_bytes": c2c_alg_bytes(n, n, n)}
    for name, kw in (("fp32_tuned", {}), ("fp32_staged_lsu", {"staged": True, "tma": False}),
                     ("fp16_split", {"precision": "fp16_split"}), ("bf16_split", {"precision": "bf16_split"}),
                     ("fp16_split_tc5", {"precision": "fp16_split_tc5"}),
                     ("bf16_split_tc5", {"precision": "bf16_split_tc5"})):
        p = gb.Plan(n, n, n, **kw)
        if name == "fp32_tuned":
            p.autotune(stream)
        med, _ = time_variant(torch, p, x, [abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE], steps, warmup, stream)
        y = p.forward(x)
        z = p.inverse(y)
        rt = float(torch.linalg.vector_norm((z.to(torch.complex128) - x.to(torch.complex128)).reshape(-1))
                   / torch.linalg.vector_norm(x.to(torch.complex128).reshape(-1)))
        del z
        w = p.forward(waves, out=y)
        peaks = w[pk[:, 2], pk[:, 1], pk[:, 0]].cpu().numpy().astype(np.complex128)
        w[pk[:, 2], pk[:, 1], pk[:, 0]] = 0
        leak = float(torch.linalg.vector_norm(w.reshape(-1).to(torch.complex128))) / float(
            np.sqrt(np.sum(np.abs(N * amps) ** 2)))
        torch.cuda.synchronize()
        out[name] = {"fwd_ms": med[0], "inv_ms": med[1],
                     "fwd_gflops": flops_5n(n, n, n) / (med[0] * 1e-3) / 1e9,
                     "fwd_alg_gbs": c2c_alg_bytes(n, n, n) / (med[0] * 1e-3) / 1e9,
                     "peak_rel_err": float(np.max(np.abs(peaks - N * amps) / np.abs(N * amps))),
                     "leak_rel": leak, "round_trip_rel_l2": rt, "device_error": p.device_error()}
        del y, w
        p.close()
    del x, waves
    torch.cuda.empty_cache()
    return out


def extra_variants(torch, gb, abi, dev, stream, steps, warmup):
    """C2C 512^3 pencil and slab, R2C slab, forward+adjoint: per-launch medians."""
    import synth
    out = {}
    x = synth.uniform_complex((N, N, N), seed=3).to(dev)
    p = gb.Plan(N, N, N)
    tz = p.autotune(stream)
    med, _ = time_variant(torch, p, x, [abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE], steps, warmup, stream)
    out["c2c_512_pencil_tuned"] = {"fwd_ms": med[0], "inv_ms": med[1], "fwd_inv_ms": med[0] + med[1],
                                   "gflops": 2 * flops_5n(N, N, N) / ((med[0] + med[1]) * 1e-3) / 1e9,
                                   "alg_gbs": 2 * c2c_alg_bytes(N, N, N) / ((med[0] + med[1]) * 1e-3) / 1e9,
                                   "frac": 2 * c2c_alg_bytes(N, N, N) / ((med[0] + med[1]) * 1e-3) / 1e9
                                   / measured_peaks()[0],
                                   "tuning": {k: {"persistent": v["persistent"], "tma_mask": v["tma_mask"]}
                                              for k, v in tz.items()}}
    p.close()
    # the persistent ticket-queue launch with the warp-per-pencil tile body on all three stages, with 1, 2 and 4
    # consecutive tiles per ticket
    pw = {}
    for log_t in (0, 1, 2):
        p = gb.Plan(N, N, N)
        for k in (0, 1):
            abi.gbfft_plan_set_tuning(p.handle, k, True, (0x7 << 20) | (log_t << 25))
        med, _ = time_variant(torch, p, x, [abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE], steps, warmup, stream)
        pw[f"tiles_per_ticket_{1 << log_t}"] = {
            "fwd_ms": med[0], "inv_ms": med[1], "fwd_inv_ms": med[0] + med[1],
            "frac": 2 * c2c_alg_bytes(N, N, N) / ((med[0] + med[1]) * 1e-3) / 1e9 / measured_peaks()[0]}
        p.close()
    out["c2c_512_persistent_warp_body"] = pw
    for slab in (False, True):
        p = gb.Plan(N, N, N, slab=slab)
        med, avg = time_variant(torch, p, x, [abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE], steps, warmup, stream)
        b = c2c_alg_bytes(N, N, N, passes=2 if slab else 3)
        key = "c2c_512_slab" if slab else "c2c_512_pencil"
        out[key] = {"fwd_ms": med[0], "inv_ms": med[1], "fwd_inv_ms": med[0] + med[1],
                    "gflops": 2 * flops_5n(N, N, N) / ((med[0] + med[1]) * 1e-3) / 1e9,
                    "alg_gbs": 2 * b / ((med[0] + med[1]) * 1e-3) / 1e9}
        p.close()
    del x
    r = synth.normal_real((N, N, N), seed=2).to(dev)
    p = gb.Plan(N, N, N, kind="r2c", slab=True)
    med, _ = time_variant(torch, p, r, [abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE], steps, warmup, stream)
    b = slab_r2c_alg_bytes(N, N, N)
    out["r2c_512_slab"] = {"fwd_ms": med[0], "inv_ms": med[1], "fwd_inv_ms": med[0] + med[1],
                           "gflops": 2 * flops_5n(N, N, N) / ((med[0] + med[1]) * 1e-3) / 1e9,
                           "alg_gbs": 2 * b / ((med[0] + med[1]) * 1e-3) / 1e9}
    p.close()
    p = gb.Plan(N, N, N, kind="r2c", slab=True)
    tz = p.autotune(stream)
    med, _ = time_variant(torch, p, r, [abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE], steps, warmup, stream)
    out["r2c_512_slab_tuned"] = {"fwd_ms": med[0], "inv_ms": med[1], "fwd_inv_ms": med[0] + med[1],
                                 "gflops": 2 * flops_5n(N, N, N) / ((med[0] + med[1]) * 1e-3) / 1e9,
                                 "alg_gbs": 2 * b / ((med[0] + med[1]) * 1e-3) / 1e9,
                                 "frac": 2 * b / ((med[0] + med[1]) * 1e-3) / 1e9 / measured_peaks()[0],
                                 "tuning": {k: {"persistent": v["persistent"], "tma_mask": v["tma_mask"] & 0xFF,
                                                "plane_mask": (v["tma_mask"] >> 8) & 0xFF,
                                                "plane_cx": (v["tma_mask"] >> 16) & 0xF} for k, v in tz.items()}}
    p.close()
    fused = {}
    for cx in (2, 4, 8):
        p = gb.Plan(N, N, N, kind="r2c", slab=True)
        abi.gbfft_plan_set_tuning(p.handle, 0, False, (1 << 8) | (cx << 16))  # x,y fused; z thread loads
        abi.gbfft_plan_set_tuning(p.handle, 1, False, (2 << 8) | (cx << 16))  # z; y,x fused
        med, _ = time_variant(torch, p, r, [abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE], steps, warmup, stream)
        fused[f"cluster_{cx}"] = {"fwd_ms": med[0], "inv_ms": med[1]}
        p.close()
    out["r2c_512_slab_fused_plane"] = fused
    # the in-plane pairs as plane launches that keep each plane's intermediate in distributed shared memory
    # (8-CTA clusters): two HBM passes per transform
    p = gb.Plan(N, N, N, kind="r2c", slab=True)
    abi.gbfft_plan_set_tuning(p.handle, 0, False, (1 << 27) | (1 << 8))  # x,y in one launch; z
    abi.gbfft_plan_set_tuning(p.handle, 1, False, (1 << 27) | (2 << 8))  # z; y,x in one launch
    med, _ = time_variant(torch, p, r, [abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE], steps, warmup, stream)
    abi.gbfft_plan_time_stages(p.handle, True)
    with torch.cuda.stream(stream):
        for _ in range(steps):
            p.inverse(p.forward(r, stream=stream), stream=stream)
    torch.cuda.synchronize()
    abi.gbfft_plan_time_stages(p.handle, False)
    seg_f, _ = abi.gbfft_plan_stage_times(p.handle, 0)
    seg_i, _ = abi.gbfft_plan_stage_times(p.handle, 1)
    pair_bytes = N * N * N * 4 + N * N * (N // 2 + 1) * 8  # real plane in, half spectrum out (or back)
    out["r2c_512_slab_dsm"] = {
        "fwd_ms": med[0], "inv_ms": med[1], "fwd_inv_ms": med[0] + med[1],
        "alg_gbs": 2 * b / ((med[0] + med[1]) * 1e-3) / 1e9,
        "frac": 2 * b / ((med[0] + med[1]) * 1e-3) / 1e9 / measured_peaks()[0],
        "launch_ms": {"forward": seg_f, "inverse": seg_i},
        "plane_launch_alg_gbs": [pair_bytes / (seg_f[0] * 1e-3) / 1e9 if seg_f else None,
                                 pair_bytes / (seg_i[1] * 1e-3) / 1e9 if len(seg_i) > 1 else None]}
    p.close()
    p = gb.Plan(N, N, N, kind="r2c")
    med, _ = time_variant(torch, p, r, [abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_ADJOINT], steps, warmup, stream)
    out["r2c_512_fwd_adjoint_ms"] = med[0] + med[1]
    p.close()
    for tma in (True, False):
        ps = gb.Plan(N, N, N, kind="r2c", staged=True, tma=tma)
        med, _ = time_variant(torch, ps, r, [abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE], steps, warmup, stream)
        out["r2c_512_pencil_staged_" + ("tma" if tma else "lsu") + "_fwd_inv_ms"] = med[0] + med[1]
        ps.close()
    x = synth.uniform_complex((N, N, N), seed=3).to(dev)
    for tma in (True, False):
        ps = gb.Plan(N, N, N, staged=True, tma=tma)
        med, _ = time_variant(torch, ps, x, [abi.GBFFT_OP_FORWARD, abi.GBFFT_OP_INVERSE], steps, warmup, stream)
        out["c2c_512_pencil_staged_" + ("tma" if tma else "lsu") + "_fwd_inv_ms"] = med[0] + med[1]
        ps.close()
    del x
    out["batched_64"] = batched_variant(torch, gb, abi, stream, steps, warmup)
    out["poisson_256"] = poisson_variant(torch, gb, abi, stream, steps, warmup)
    out["precision_1024"] = precision_variant(torch, gb, abi, stream, min(steps, 10), warmup)
    # cuFFT via torch.fft on the same GPU: context only, not a target
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(warmup):
        torch.fft.irfftn(torch.fft.rfftn(r), s=(N, N, N))
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(steps):
        torch.fft.irfftn(torch.fft.rfftn(r), s=(N, N, N))
    ev1.record()
    torch.cuda.synchronize()
    out["context_torch_fft_r2c_c2r_ms"] = ev0.elapsed_time(ev1) / steps
    return out


if __name__ == "__main__":
    main()
