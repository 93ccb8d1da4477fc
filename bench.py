"""Throughput of dense membrane-probability inference (Sec. 2.1-2.2) on one GB300.

One step = one pass of the inference path over the 1024x1024x32 uint8 synthetic EM volume
(32 independent slices, the generator's 120 cells per 256^2): every pixel's probability map.
`value` is output megavoxels per second with the volume resident in HBM; `e2e` is the same
metric through the C ABI with pinned HOST buffers (host<->device copies inside the timed region).
L2 is flushed (a 256 MB write) between timed steps. The reference arm is the FP64 CPU oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16|fp32|fp8] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "membrane-prob megavoxels/s on 1 GB300: FP32 vs BF16/FP8 vs student, at stated error"
Z, H, W = 32, 1024, 1024
WORKLOAD = "1024x1024x32 uint8 synthetic EM volume (32 independent slices), stand-in teacher CNN"
FLOP_PER_PX = 2 * (25 * 32 + 2 * 25 * 32 * 32 + 32)        # 104,064
TENSOR_FLOP_PER_PX = 2 * 2 * 25 * 32 * 32                   # 102,400 (layers 2 and 3)
BYTES_PER_PX = {0: 5, 1: 2}                                 # 1 B in + 4 B (float) or 1 B (u8) out


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not self.path:
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(params, vol, budget_s=20.0):
    """The FP64 oracle as it stands, on a bounded sample: 256x256 crops (true context) of
    successive slices until about budget_s of CPU time."""
    import oracle
    import synth
    t0 = time.perf_counter()
    n = 0
    while True:
        zi = n % vol.shape[0]
        oracle.forward_region(synth.TEACHER, params, vol[zi], 384, 384, 256, 256)
        n += 1
        if time.perf_counter() - t0 > budget_s or n >= 64:
            break
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n * 256 * 256 / dt / 1e6, "unit": "Mvox/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} crops of 256x256 (7-px true context) from slices of the 1024x1024x32 volume, "
                      f"FP64 direct loops, {dt:.1f} s"}


def run_reference(args):
    import numpy as np  # noqa: F401
    import synth
    params = synth.init_params(synth.TEACHER, synth.TEACHER_WEIGHT_SEED)
    vol = synth.em_volume(synth.BASE_SEED + 1, 4, H, W)
    import oracle
    crop = 256

    def step(i):
        oracle.forward_region(synth.TEACHER, params, vol[i % 4], 384, 384, crop, crop)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(i)
    dt = time.perf_counter() - t0
    value = args.steps * crop * crop / dt / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mvox/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64-oracle"},
            "cpu_baseline": {"value": value, "unit": "Mvox/s", "cores": cores, "kind": "oracle",
                             "sample": f"one 256x256 crop (true context) per step, FP64 direct loops"},
            "e2e": {"value": value, "unit": "Mvox/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["fp32", "bf16", "fp8"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--extra", action="store_true", help="also time the other precision paths")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import numpy as np
    import torch

    import synth
    from paper_1612_02120_gb300 import build as pbuild
    from paper_1612_02120_gb300 import membrane as m

    if rank == 0:
        pbuild.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        if rank != 0:
            pbuild.build()

    prec = {"fp32": m.MB_PREC_FP32, "bf16": m.MB_PREC_BF16, "fp8": m.MB_PREC_FP8}[args.prec]
    params = synth.init_params(synth.TEACHER, synth.TEACHER_WEIGHT_SEED)
    vol = synth.em_volume(synth.BASE_SEED + 1, Z, H, W)
    x = torch.from_numpy(vol).cuda()
    out = torch.empty((Z, H, W), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()

    net = m.Net(synth.TEACHER, prec, local, params)
    if prec == m.MB_PREC_FP8:
        m.mb_calibrate_fp8(net.handle, x[:4], 4, H, W, stream=stream)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            m.mb_infer_volume(net.handle, x, Z, H, W, out, m.MB_OUT_F32, stream)
        barrier()
        launches0 = m.launch_count()
        times = []
        with ClockSampler(local) as clk:
            for _ in range(args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                m.mb_infer_volume(net.handle, x, Z, H, W, out, m.MB_OUT_F32, stream)
                e1.record(stream)
                times.append((e0, e1))
            torch.cuda.synchronize()
        launches = m.launch_count() - launches0
        step_ms = [a.elapsed_time(b) for a, b in times]
    total_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        barrier()
    ms_per_step = total_ms / args.steps
    vox = Z * H * W
    value = world * vox / (ms_per_step / 1e3) / 1e6

    # end to end through the C ABI with pinned host buffers
    pin_in = torch.from_numpy(vol).pin_memory()
    pin_out = torch.empty((Z, H, W), dtype=torch.float32).pin_memory()
    m.mb_infer_volume(net.handle, pin_in, Z, H, W, pin_out)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        m.mb_infer_volume(net.handle, pin_in, Z, H, W, pin_out)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_value = world * vox / e2e_s / 1e6

    pk, pk_kind = peaks()
    kernel_ms = statistics.mean(step_ms)
    if prec == m.MB_PREC_FP32:
        sm_mhz = pk.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        achieved = FLOP_PER_PX * vox / (kernel_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "conv_simt (3 launches per step, all layers)",
                "peak_kind": "derived: 152 SMs x 128 FP32 FMA/clk x 2 x max SM clock"}
    else:
        peak = pk["bf16_tflops_sustained"] if prec == m.MB_PREC_BF16 else 2 * pk["bf16_tflops_sustained"]
        achieved = TENSOR_FLOP_PER_PX * vox / (kernel_ms / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "tc_fused_teacher (1 launch per step)",
                "peak_kind": f"{pk_kind} bf16 sustained" + (" x 2 (nominal fp8/bf16 ratio)" if prec == m.MB_PREC_FP8 else "")}

    line = {"metric": METRIC, "value": value, "unit": "Mvox/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "fp8e4m3"}[args.prec],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": args.prec, "out": "float32",
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas{world}"},
            "gb_per_hour": value * 1e6 * 3600 / 1e9,
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": "Mvox/s", "h2d_bytes_per_step": vox, "d2h_bytes_per_step": 4 * vox},
            "gpu_launches": launches,
            "clocks": clk.summary()}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(params, vol)
    net.close()
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
