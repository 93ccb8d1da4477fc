"""Throughput of dense membrane-probability inference (Sec. 2.1-2.2) on one GB300.

Headline step: one pass of the BF16 tensor-core path over the 1024x1024x32 uint8 synthetic EM
volume (32 independent slices; 120 Voronoi cells per 256^2, membranes 2-3 px, blur sigma 1), every
pixel's probability map. `value` = output megavoxels/s with the volume resident in HBM; `e2e` =
the same through the C ABI with pinned HOST buffers (the kernel reads the input from and writes the
maps to host memory inside the timed region; the slab mode, copies through device buffers, is
timed beside it). L2 is flushed
(256 MB write) between timed steps. The same run measures, under "paths":
  cfg1  FP32 / BF16 / FP8 on the same volume, each with max-abs, mean-abs, agreement at 0.5 and
        near-threshold mass against the FP64 oracle on 2 seeded slices;
  cfg2  64 uneven blocks (sides U[256,1536], depth U[1,16]) BF16: one persistent launch under a
        captured CUDA graph (autotuned on the batch) vs one launch per block;
  cfg3  4096x4096x64 FP8 (calibrated on 4 slices) and BF16, resident and from pinned host
        memory; errors on 3 seeded 512x512 crops (true context);
  cfg4  student training (200 x 512^2, batch 32, lr 1e-3, 2000 steps) on FP32-teacher maps, then
        student-only and cascade (teacher fallback on 256^2 tiles) on the cfg3 volume;
  cfg8  the second teacher workload: the stand-in with its head fitted to the generator's membrane
        truth (a map that straddles 0.5): FP32/BF16/FP8 errors and accuracy against the truth, a
        student distilled from it, and the cascade under the stated rule on the cfg3 volume;
  cfg6  FastMemb_3nm (one more stage, 109 field of view) on 2048x2048x8 (3 nm images), FP32,
        BF16 and FP16, dense and sub-sampled by 2 (a 6 nm output map), errors on 2 seeded 256x256 crops;
  cfg7  MaskExtend (Sec. 3.2): the +z transfer recursion on a 512x512 window for 16 sections
        (FP32), errors of one step's 3 class maps against the oracle on a 128x128 crop;
  cfg5  FastMemb in dense form (Sec. 2.2) on the cfg1 volume, FP32, BF16 and FP16, dense and sub-sampled
        by 2 (the pruned fragment tree), with errors against the oracle on 3 seeded 384x384 crops
        (true context; even crop origins, so the sub-sampled crops are the dense crops' even pixels).
The reference arm (--impl reference) is the FP64 CPU oracle on bounded samples.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--configs 1,2,3,4]
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
sys.path.insert(0, ROOT)

METRIC = "membrane-prob megavoxels/s on 1 GB300: FP32 vs BF16/FP8 vs student, at stated error"
Z, H, W = 32, 1024, 1024
WORKLOAD = "1024x1024x32 uint8 synthetic EM volume (32 independent slices), stand-in teacher CNN, BF16"
FLOP_PER_PX = 2 * (25 * 32 + 2 * 25 * 32 * 32 + 32)        # 104,064
TENSOR_FLOP_PER_PX = 2 * 2 * 25 * 32 * 32                   # 102,400 (layers 2 and 3)
STUDENT_FLOP_PER_PX = 2 * (9 * 16 + 9 * 16 * 16 + 16)       # 4,928
FASTMEMB_FLOP_PER_PX = 2 * (16 * 64 + 2 * 16 * 32 * 64 + 16 * 32 * 2)  # 135,168
FASTMEMB3_FLOP_PER_PX = 2 * (16 * 64 + 3 * 16 * 32 * 64 + 16 * 32 * 2)  # 200,704
MASKEXTEND_FLOP_PER_PX = 2 * (16 * 12 * 64 + 16 * 32 * 80 + 16 * 40 * 96 + 16 * 48 * 112 + 16 * 56 * 128 + 64 * 3)
# Sources of the headline kernel: a DRAM-traffic record taken by ncu is used only while these
# files hash to the value recorded with it (otherwise the kernel changed since the capture).
TC_SOURCES = ("paper_1612_02120_gb300/csrc/tc_conv.cu", "paper_1612_02120_gb300/csrc/tc_ptx.cuh",
              "paper_1612_02120_gb300/csrc/internal.h")
TC_TRAFFIC_RECORD = "profiles/tc_fused_teacher_bf16_1024x1024x32.traffic.txt"
TOL = {"fp32": {"max_abs": 1e-5}, "bf16": {"max_abs": 3e-2, "mean_abs": 2e-3},
       "fp8": {"max_abs": 1e-1, "mean_abs": 1e-2}, "student": {"mean_abs": 3e-2}}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples every 25 ms during a timed region. The region starts only once the
    sampler has written its first sample (nvidia-smi takes a while to start), so that the samples
    fall inside it."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu, self.proc, self.path = gpu_index, None, None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 3.0 and self.proc.poll() is None and os.path.getsize(self.path) == 0:
                time.sleep(0.01)
            self.f.flush()
            self.skip = os.path.getsize(self.path)  # bytes written before the timed region
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
        with open(self.path) as fh:
            text = fh.read()
        os.unlink(self.path)
        skip = min(getattr(self, "skip", 0), len(text))

        def parse(t):
            rows = [[p.strip() for p in line.split(",")] for line in t.splitlines()]
            return [r for r in rows if len(r) >= 9]
        rows = parse(text[skip:])
        in_region = len(rows)
        if not rows:  # a region shorter than one sampling interval: the sample taken just before it
            rows = parse(text[:skip])
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [v for v in (num(r[1]) for r in rows) if v is not None]
        mx = [v for v in (num(r[2]) for r in rows) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": in_region}


def cpu_cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def kernel_source_hash(paths=TC_SOURCES):
    import hashlib
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(path=TC_TRAFFIC_RECORD):
    """(bytes per launch, note) from an ncu record of `key value` lines, or (None, why) when the
    record is missing or was taken on other kernel sources."""
    try:
        with open(os.path.join(ROOT, path)) as f:
            rec = dict(line.split(None, 1) for line in f.read().splitlines() if line.strip() and " " in line)
    except OSError:
        return None, "no ncu traffic record"
    want = kernel_source_hash()
    if rec.get("source_sha256_16", "").strip() != want:
        return None, f"kernel sources changed since the ncu capture (now {want})"
    return float(rec["dram_bytes_per_launch"]), rec.get("captured", "").strip()


def oracle_rate(budget_s, crop=256, max_crops=64):
    """Mvox/s of the FP64 oracle as it stands on crops (true context) of successive slices of the
    headline volume, until about budget_s; returns (value, crops, seconds)."""
    import oracle
    import synth
    params = synth.init_params(synth.TEACHER, synth.TEACHER_WEIGHT_SEED)
    vol = synth.em_volume(synth.BASE_SEED + 1, 4, H, W)
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle.forward_region(synth.TEACHER, params, vol[n % vol.shape[0]], 384, 384, crop, crop)
        n += 1
        if time.perf_counter() - t0 > budget_s or n >= max_crops:
            break
    dt = time.perf_counter() - t0
    return n * crop * crop / dt / 1e6, n, dt


def cpu_baseline(budget_s=12.0, single_budget_s=10.0):
    """The FP64 oracle as it stands on a bounded sample, on all host cores and on one thread (a
    child process with OMP_NUM_THREADS=1: the thread count is fixed when OpenMP starts)."""
    v, n, dt = oracle_rate(budget_s)
    out = {"value": v, "unit": "Mvox/s", "cores": cpu_cores(), "kind": "oracle",
           "sample": f"{n} crops of 256x256 (7-px true context) of the 1024x1024 headline slices, FP64 direct "
                     f"loops, {dt:.1f} s"}
    try:
        env = dict(os.environ, OMP_NUM_THREADS="1")
        code = (f"import json, bench; v, n, dt = bench.oracle_rate({single_budget_s}); "
                "print(json.dumps([v, n, dt]))")
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=single_budget_s + 120)
        v1, n1, dt1 = json.loads(r.stdout.strip().splitlines()[-1])
        out["single_thread"] = {"value": v1, "unit": "Mvox/s", "cores": 1,
                                "sample": f"{n1} crops of 256x256 (true context), {dt1:.1f} s"}
        out["parallel_speedup"] = v / v1
    except Exception as e:  # reported, never fatal for the bench line
        out["single_thread"] = {"unavailable": f"{type(e).__name__}: {e}"[:200]}
    return out


def run_reference(args):
    import oracle
    import synth
    params = synth.init_params(synth.TEACHER, synth.TEACHER_WEIGHT_SEED)
    vol = synth.em_volume(synth.BASE_SEED + 1, 4, H, W)
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
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mvox/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "fp64-oracle"},
        "cpu_baseline": {"value": value, "unit": "Mvox/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": "one 256x256 crop (true context) of a 1024x1024 slice per step, FP64"},
        "e2e": {"value": value, "unit": "Mvox/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def truth_head_fixture():
    with open(os.path.join(ROOT, "tests", "golden", "truth_head.json")) as f:
        return json.load(f)


def truth_head_params(params):
    """The second teacher workload: the stand-in's layers 1-3 with the head fitted to the
    generator's membrane truth (a stored fixture written from the FP64 oracle's features)."""
    import numpy as np
    fx = truth_head_fixture()
    p = np.array(params, dtype=np.float32, copy=True)
    p[-33:-1] = np.asarray(fx["head_w"], dtype=np.float32)
    p[-1] = np.float32(fx["head_b"])
    return p


def truth_accuracy(maps, truths):
    """Fraction of pixels where (p >= 0.5) equals the generator's membrane flag."""
    import numpy as np
    a = np.concatenate([np.asarray(m).ravel() >= 0.5 for m in maps])
    t = np.concatenate([np.asarray(x).ravel() > 0 for x in truths])
    return float((a == t).mean())


def max_over_ranks(x, dist, device="cuda"):
    """This rank's time -> the maximum over all ranks (the whole job finishes with its slowest
    rank); unchanged on a single process."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mvox_s(world, vox_per_rank, seconds):
    """Whole-job throughput: every rank processed vox_per_rank voxels (weak scaling, replicas)."""
    return world * vox_per_rank / seconds / 1e6


def time_device(fn, steps, warmup, stream, flush):
    """Per-step CUDA-event times (ms) of fn() on `stream`, L2 flushed between steps."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def err_metrics(maps, refs, tol):
    import numpy as np
    import oracle
    a = np.concatenate([np.asarray(m, dtype=np.float64).ravel() for m in maps])
    r = np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in refs])
    met = oracle.metrics(a, r)
    met["within_tolerance"] = all((met[k] <= v) for k, v in tol.items()) and met["agreement"] >= 0.995
    return met


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--configs", default="1,2,3,4,8,5,6,7", help="extra configurations measured after the headline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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

    import oracle
    import synth
    from paper_1612_02120_gb300 import build as pbuild
    from paper_1612_02120_gb300 import membrane as m

    pbuild.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    params = synth.init_params(synth.TEACHER, synth.TEACHER_WEIGHT_SEED)
    vol = synth.em_volume(synth.BASE_SEED + 1, Z, H, W)
    x = torch.from_numpy(vol).cuda()
    out = torch.empty((Z, H, W), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    vox = Z * H * W

    # ---- headline: BF16 fused tensor-core kernel on cfg1 ------------------------------------------
    net = m.Net(synth.TEACHER, m.MB_PREC_BF16, local, params)
    # the library's autotuner picks rows per work item and pipeline lag for this shape (cached)
    tune_cache = os.path.join(tempfile.gettempdir(), "membrane_tune.json")
    head_tune = m.mb_autotune(net.handle, Z, H, W, tune_cache, stream)
    with torch.cuda.stream(stream):
        def step():
            m.mb_infer_volume(net.handle, x, Z, H, W, out, m.MB_OUT_F32, stream)
        for _ in range(args.warmup):
            step()
        barrier()
        launches0 = m.launch_count()
        with ClockSampler(local) as clk:
            step_ms = time_device(step, args.steps, 0, stream, flush)
        launches = m.launch_count() - launches0
    total_ms = max_over_ranks(sum(step_ms), dist)
    barrier()
    ms_per_step = total_ms / args.steps
    value = whole_job_mvox_s(world, vox, ms_per_step / 1e3)
    bf16_map = out.cpu().numpy()

    # end to end through the C ABI with pinned host buffers: in the default host I/O mode the
    # kernel itself loads the input from and stores the maps to the pinned buffers over the
    # coherent CPU-GPU link; the slab mode (copies through device buffers) is timed beside it
    pin_in = torch.from_numpy(vol).pin_memory()
    pin_out = torch.empty((Z, H, W), dtype=torch.float32, pin_memory=True)

    def e2e_leg(mode):
        m.mb_set_host_io(net.handle, mode)
        m.mb_infer_volume(net.handle, pin_in, Z, H, W, pin_out)
        barrier()
        n0 = m.launch_count()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            m.mb_infer_volume(net.handle, pin_in, Z, H, W, pin_out)
        secs = max_over_ranks((time.perf_counter() - t0) / args.steps, dist)
        return whole_job_mvox_s(world, vox, secs), (m.launch_count() - n0) / args.steps

    e2e_slabs, slab_launches = e2e_leg(m.MB_HOST_IO_SLABS)
    e2e_value, e2e_launches = e2e_leg(m.MB_HOST_IO_AUTO)
    e2e_exact = np.array_equal(pin_out.numpy(), bf16_map)
    e2e_io = ("direct: the fused kernel loads the pinned input and stores the pinned maps over the "
              "CPU-GPU link, one launch per call" if e2e_launches == 1 else
              "slabs: copies through device buffers overlapped with compute")

    pk, pk_kind = peaks()
    kernel_ms = statistics.mean(step_ms)
    achieved = TENSOR_FLOP_PER_PX * vox / (kernel_ms / 1e3) / 1e12
    # the timed region is K launches of a few ms each (well under a second): the burst peak applies
    peak = pk["bf16_tflops"]
    traffic, traffic_note = recorded_traffic()
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_source": traffic_note,
            "algorithmic_bytes": 5 * vox,
            "kernel": "tc_fused_teacher<bf16> (1 launch per step)",
            "algorithmic": f"{TENSOR_FLOP_PER_PX} tensor FLOP/px x {vox} px per launch; "
                           f"{FLOP_PER_PX} FLOP/px in all; 5 B/px of DRAM",
            "peak_kind": f"{pk_kind} bf16 dense, burst (timed region {sum(step_ms):.0f} ms)",
            "frac_of_sustained": achieved / pk["bf16_tflops_sustained"],
            "hbm_frac": 5 * vox / (kernel_ms / 1e3) / 1e9 / pk["hbm_gbs"]}

    line = {"metric": METRIC, "value": value, "unit": "Mvox/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "bf16 (layers 2-3), fp32 (layer 1, head)",
                       "out": "float32", "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"replicas{world}"},
            "gb_per_hour": value * 1e6 * 3600 / 1e9, "roofline": roof, "autotune": head_tune,
            "e2e": {"value": e2e_value, "unit": "Mvox/s", "h2d_bytes_per_step": vox, "d2h_bytes_per_step": 4 * vox,
                    "host_io": e2e_io, "launches_per_call": e2e_launches, "equals_device_maps": bool(e2e_exact),
                    "slabs": {"value": e2e_slabs, "launches_per_call": slab_launches}},
            "gpu_launches": launches, "clocks": clk.summary()}
    configs = {c.strip() for c in args.configs.split(",") if c.strip()} if world == 1 else set()
    paths = {}

    # ---- cfg1: FP32 / BF16 / FP8 on the same volume + errors on 2 seeded slices --------------------
    if "1" in configs:
        zs = [int(z) for z in np.random.default_rng(synth.BASE_SEED + 1).choice(Z, 2, replace=False)]
        refs = [oracle.forward_region(synth.TEACHER, params, vol[z]) for z in zs]
        p = {"bf16": {"mvox_s": value, "ms": ms_per_step,
                      "error": err_metrics([bf16_map[z] for z in zs], refs, TOL["bf16"])}}
        # uint8 output (q = round(255 p)): 1 B/vox stored instead of 4, through the same kernel
        out_u8 = torch.empty((Z, H, W), dtype=torch.uint8, device="cuda")
        with torch.cuda.stream(stream):
            ms = time_device(lambda: m.mb_infer_volume(net.handle, x, Z, H, W, out_u8, m.MB_OUT_U8, stream),
                             args.steps, 3, stream, flush)
        p["bf16_u8_out"] = {"mvox_s": vox / (statistics.mean(ms) / 1e3) / 1e6, "ms": statistics.mean(ms)}
        del out_u8
        fp32 = m.Net(synth.TEACHER, m.MB_PREC_FP32, local, params)
        with torch.cuda.stream(stream):
            ms = time_device(lambda: m.mb_infer_volume(fp32.handle, x, Z, H, W, out, m.MB_OUT_F32, stream),
                             3, 1, stream, flush)
        p["fp32"] = {"mvox_s": vox / (statistics.mean(ms) / 1e3) / 1e6, "ms": statistics.mean(ms),
                     "error": err_metrics([out[z].cpu().numpy() for z in zs], refs, TOL["fp32"])}
        fp32.close()
        fp8 = m.Net(synth.TEACHER, m.MB_PREC_FP8, local, params)
        m.mb_calibrate_fp8(fp8.handle, x[:4], 4, H, W, stream=stream)
        m.mb_autotune(fp8.handle, Z, H, W, tune_cache, stream)
        with torch.cuda.stream(stream):
            ms = time_device(lambda: m.mb_infer_volume(fp8.handle, x, Z, H, W, out, m.MB_OUT_F32, stream),
                             args.steps, 3, stream, flush)
        p["fp8"] = {"mvox_s": vox / (statistics.mean(ms) / 1e3) / 1e6, "ms": statistics.mean(ms),
                    "error": err_metrics([out[z].cpu().numpy() for z in zs], refs, TOL["fp8"])}
        fp8.close()
        for k in ("bf16", "fp8"):
            p[k]["speedup_vs_fp32"] = p[k]["mvox_s"] / p["fp32"]["mvox_s"]
        p["sampled_slices"] = zs
        paths["cfg1_1024x1024x32"] = p

    # ---- cfg2: 64 uneven blocks, persistent launch + graph vs per-block launches --------------------
    if "2" in configs:
        shapes = synth.block_shapes(synth.BASE_SEED + 2, 64)
        ins, outs, blocks = [], [], []
        for i, (d, h, w) in enumerate(shapes):
            v = torch.from_numpy(synth.em_volume(synth.BASE_SEED + 2, d, h, w, block=i)).cuda()
            o = torch.empty((d, h, w), dtype=torch.float32, device="cuda")
            ins.append(v)
            outs.append(o)
            blocks.append((v, d, h, w, w, h * w, o, w, h * w))
        bvox = sum(d * h * w for d, h, w in shapes)
        # tuned on the batch itself (a single-volume tuning shape does not predict the uneven blocks'
        # best schedule; it picked 128-row items here where the even split is 8 % faster)
        tune = m.mb_autotune_batch(net.handle, blocks, m.MB_OUT_F32, tune_cache, stream)
        with torch.cuda.stream(stream):
            ms_b = time_device(lambda: m.mb_infer_batch(net.handle, blocks, m.MB_OUT_F32, stream), args.steps, 3,
                               stream, flush)
            l0 = m.launch_count()
            m.mb_infer_batch(net.handle, blocks, m.MB_OUT_F32, stream)
            lb = m.launch_count() - l0
            ms_p = time_device(lambda: m.mb_infer_batch_per_block(net.handle, blocks, m.MB_OUT_F32, stream),
                               args.steps, 3, stream, flush)
        paths["cfg2_64_uneven_blocks"] = {
            "voxels": bvox, "persistent_graph_mvox_s": bvox / (statistics.mean(ms_b) / 1e3) / 1e6,
            "per_block_mvox_s": bvox / (statistics.mean(ms_p) / 1e3) / 1e6,
            "speedup": statistics.mean(ms_p) / statistics.mean(ms_b), "launches_per_batch": lb,
            "autotune": tune}

    # ---- cfg3: 4096x4096x64, FP8 and BF16, resident and streamed --------------------------------
    big = None
    if "3" in configs or "4" in configs or "8" in configs:
        Z3, H3, W3 = 64, 4096, 4096
        big = torch.empty((Z3, H3, W3), dtype=torch.uint8, pin_memory=True)
        synth.em_volume(synth.BASE_SEED + 3, Z3, H3, W3, out=big.numpy())
        xb = big.cuda()
        ob = torch.empty((Z3, H3, W3), dtype=torch.float32, device="cuda")
        v3 = Z3 * H3 * W3
        rng = np.random.default_rng(synth.BASE_SEED + 3)
        crops = [(int(rng.integers(Z3)), int(rng.integers(H3 - 512)), int(rng.integers(W3 - 512))) for _ in range(3)]
        crop_refs = [oracle.forward_region(synth.TEACHER, params, big[z].numpy(), y, x0, 512, 512)
                     for z, y, x0 in crops]
    if "3" in configs:
        p = {}
        for name, prec in (("fp8", m.MB_PREC_FP8), ("bf16", m.MB_PREC_BF16)):
            n3 = m.Net(synth.TEACHER, prec, local, params)
            if prec == m.MB_PREC_FP8:
                m.mb_calibrate_fp8(n3.handle, xb[:4], 4, H3, W3, stream=stream)
            m.mb_autotune(n3.handle, 4, H3, W3, tune_cache, stream)
            with torch.cuda.stream(stream):
                ms = time_device(lambda: m.mb_infer_volume(n3.handle, xb, Z3, H3, W3, ob, m.MB_OUT_F32, stream),
                                 3, 1, stream, flush)
            err = err_metrics([ob[z, y:y + 512, x0:x0 + 512].cpu().numpy() for z, y, x0 in crops], crop_refs,
                              TOL[name])
            entry = {"mvox_s": v3 / (statistics.mean(ms) / 1e3) / 1e6, "ms": statistics.mean(ms), "error": err}
            if prec == m.MB_PREC_FP8:
                # 1 GB in, 4 GB out in pinned host memory: kernel-direct access, then slabs
                pin_o = torch.empty((Z3, H3, W3), dtype=torch.float32, pin_memory=True)
                for key, mode in (("host_direct_mvox_s", m.MB_HOST_IO_AUTO), ("streamed_mvox_s", m.MB_HOST_IO_SLABS)):
                    m.mb_set_host_io(n3.handle, mode)
                    m.mb_infer_volume(n3.handle, big, Z3, H3, W3, pin_o)  # warm-up (the slab buffers)
                    t0 = time.perf_counter()
                    for _ in range(2):
                        m.mb_infer_volume(n3.handle, big, Z3, H3, W3, pin_o)
                    entry[key] = 2 * v3 / (time.perf_counter() - t0) / 1e6
                del pin_o
            p[name] = entry
            n3.close()
        p["fp8"]["speedup_vs_bf16"] = p["fp8"]["mvox_s"] / p["bf16"]["mvox_s"]
        p["crops"] = crops
        paths["cfg3_4096x4096x64"] = p

    # ---- cfg4: student training, student-only and cascade inference ------------------------------
    if "4" in configs:
        n_tr, s_tr = 200, 512
        tv = torch.from_numpy(synth.em_volume(synth.BASE_SEED + 4, n_tr, s_tr, s_tr)).cuda()
        tgt = torch.empty((n_tr, s_tr, s_tr), dtype=torch.float32, device="cuda")
        teacher32 = m.Net(synth.TEACHER, m.MB_PREC_FP32, local, params)
        m.mb_infer_volume(teacher32.handle, tv, n_tr, s_tr, s_tr, tgt)
        teacher32.close()
        sp = synth.init_params(synth.STUDENT, synth.STUDENT_WEIGHT_SEED, bias_std=0.0, centred_input=True)
        student = m.Net(synth.STUDENT, m.MB_PREC_BF16, local, sp)
        untrained = m.Net(synth.STUDENT, m.MB_PREC_BF16, local, sp)
        cfg = m.train_cfg(batch=32, steps=2000, lr=1e-3, seed=synth.BASE_SEED + 4)
        curve = np.zeros(2000, dtype=np.float32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.mb_student_train(student.handle, tv, tgt, n_tr, s_tr, s_tr, cfg, None, curve)
        train_s = time.perf_counter() - t0
        del tv, tgt
        Z3, H3, W3 = 64, 4096, 4096
        v3 = Z3 * H3 * W3
        with torch.cuda.stream(stream):
            ms_s = time_device(lambda: m.mb_infer_volume(student.handle, xb, Z3, H3, W3, ob, m.MB_OUT_F32, stream),
                               3, 1, stream, flush)
        s_map = [ob[z, y:y + 512, x0:x0 + 512].cpu().numpy() for z, y, x0 in crops]
        m.mb_infer_volume(untrained.handle, xb, Z3, H3, W3, ob, m.MB_OUT_F32, stream)
        torch.cuda.synchronize()
        u_map = [ob[z, y:y + 512, x0:x0 + 512].cpu().numpy() for z, y, x0 in crops]
        teacher = m.Net(synth.TEACHER, m.MB_PREC_BF16, local, params)
        m.mb_infer_volume(teacher.handle, xb, Z3, H3, W3, ob, m.MB_OUT_F32, stream)
        torch.cuda.synchronize()
        t_map = [ob[z, y:y + 512, x0:x0 + 512].cpu().numpy() for z, y, x0 in crops]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rate = m.mb_infer_cascade(student.handle, teacher.handle, xb, Z3, H3, W3, ob, 256, 0.3, 0.7, 0.05,
                                  stream=stream)
        casc_s = time.perf_counter() - t0
        c_map = [ob[z, y:y + 512, x0:x0 + 512].cpu().numpy() for z, y, x0 in crops]
        # a second reading of "ambiguous": bands of half-width 0.02 .. 0.05 around the 0.5 decision
        # threshold (the stated band holds nearly every output of this teacher); the sweep gives the
        # trade-off between the fallback rate, the speed and the agreement
        bands = []
        for hw in (0.02, 0.03, 0.04, 0.05):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = m.mb_infer_cascade(student.handle, teacher.handle, xb, Z3, H3, W3, ob, 256, 0.5 - hw, 0.5 + hw,
                                   0.05, stream=stream)
            dt = time.perf_counter() - t0
            b_map = [ob[z, y:y + 512, x0:x0 + 512].cpu().numpy() for z, y, x0 in crops]
            bands.append({"band": [0.5 - hw, 0.5 + hw], "tile": 256, "max_frac": 0.05, "fallback_rate": r,
                          "mvox_s": v3 / dt / 1e6, "vs_teacher": err_metrics(b_map, t_map, TOL["student"]),
                          "vs_oracle": err_metrics(b_map, crop_refs, TOL["student"])})
        paths["cfg4_student"] = {
            "train": {"steps": 2000, "batch": 32, "slices": n_tr, "seconds": train_s, "steps_per_s": 2000 / train_s,
                      "loss_first10": float(curve[:10].mean()), "loss_last10": float(curve[-10:].mean())},
            "student_only_mvox_s": v3 / (statistics.mean(ms_s) / 1e3) / 1e6,
            "student_tflops": STUDENT_FLOP_PER_PX * v3 / (statistics.mean(ms_s) / 1e3) / 1e12,
            "student_vs_teacher": err_metrics(s_map, t_map, TOL["student"]),
            "student_vs_oracle": err_metrics(s_map, crop_refs, TOL["student"]),
            "untrained_vs_teacher": err_metrics(u_map, t_map, TOL["student"]),
            "cascade": {"band": [0.3, 0.7], "tile": 256, "max_frac": 0.05, "fallback_rate": rate,
                        "mvox_s": v3 / casc_s / 1e6,
                        "vs_teacher": err_metrics(c_map, t_map, TOL["student"]),
                        "vs_oracle": err_metrics(c_map, crop_refs, TOL["student"])},
            "cascade_threshold_bands": bands}
        student.close()
        untrained.close()
        teacher.close()
    # ---- cfg8: the second teacher workload, a head fitted to the generator's membrane truth ------
    if "8" in configs:
        tparams = truth_head_params(params)
        p8 = {"head": "stand-in layers 1-3, head fitted to the generator's membrane flag (L2 logistic "
                      "regression, held-out accuracy %.4f)" % truth_head_fixture()["held_out_accuracy"]}
        zs = [int(z) for z in np.random.default_rng(synth.BASE_SEED + 8).choice(Z, 2, replace=False)]
        truth = [synth.em_slice_truth(synth.slice_seed(synth.BASE_SEED + 1, 0, z), H, W)[1] for z in zs]
        refs = [oracle.forward_region(synth.TEACHER, tparams, vol[z]) for z in zs]
        p8["oracle_accuracy_vs_truth"] = truth_accuracy(refs, truth)
        t_ms = {}
        for name, prec in (("fp32", m.MB_PREC_FP32), ("bf16", m.MB_PREC_BF16), ("fp8", m.MB_PREC_FP8)):
            n8 = m.Net(synth.TEACHER, prec, local, tparams)
            if prec == m.MB_PREC_FP8:
                m.mb_calibrate_fp8(n8.handle, x[:4], 4, H, W, stream=stream)
            k, w0 = (3, 1) if prec == m.MB_PREC_FP32 else (args.steps, 3)
            with torch.cuda.stream(stream):
                ms = time_device(lambda: m.mb_infer_volume(n8.handle, x, Z, H, W, out, m.MB_OUT_F32, stream), k, w0,
                                 stream, flush)
            got = [out[z].cpu().numpy() for z in zs]
            t_ms[name] = statistics.mean(ms)
            p8[name] = {"mvox_s": vox / (t_ms[name] / 1e3) / 1e6, "error": err_metrics(got, refs, TOL[name]),
                        "accuracy_vs_truth": truth_accuracy(got, truth)}
            n8.close()
        p8["slices_1024"] = zs
        # the student distilled from this teacher's FP32 maps (the configuration's training recipe)
        n_tr, s_tr = 200, 512
        tv = torch.from_numpy(synth.em_volume(synth.BASE_SEED + 4, n_tr, s_tr, s_tr)).cuda()
        tgt = torch.empty((n_tr, s_tr, s_tr), dtype=torch.float32, device="cuda")
        with m.Net(synth.TEACHER, m.MB_PREC_FP32, local, tparams) as t32:
            m.mb_infer_volume(t32.handle, tv, n_tr, s_tr, s_tr, tgt)
        sp = synth.init_params(synth.STUDENT, synth.STUDENT_WEIGHT_SEED, bias_std=0.0, centred_input=True)
        student = m.Net(synth.STUDENT, m.MB_PREC_BF16, local, sp)
        curve = np.zeros(2000, dtype=np.float32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.mb_student_train(student.handle, tv, tgt, n_tr, s_tr, s_tr,
                           m.train_cfg(batch=32, steps=2000, lr=1e-3, seed=synth.BASE_SEED + 4), None, curve)
        p8["train"] = {"seconds": time.perf_counter() - t0, "loss_first10": float(curve[:10].mean()),
                       "loss_last10": float(curve[-10:].mean())}
        del tv, tgt
        Z3, H3, W3 = 64, 4096, 4096
        v3 = Z3 * H3 * W3
        c_truth = [synth.em_slice_truth(synth.slice_seed(synth.BASE_SEED + 3, 0, z), H3, W3)[1][y:y + 512, x0:x0 + 512]
                   for z, y, x0 in crops]
        c_refs = [oracle.forward_region(synth.TEACHER, tparams, big[z].numpy(), y, x0, 512, 512) for z, y, x0 in crops]

        def crops_of(t):
            return [t[z, y:y + 512, x0:x0 + 512].cpu().numpy() for z, y, x0 in crops]
        teacher = m.Net(synth.TEACHER, m.MB_PREC_BF16, local, tparams)
        m.mb_autotune(teacher.handle, 4, H3, W3, tune_cache, stream)
        with torch.cuda.stream(stream):
            ms_t = time_device(lambda: m.mb_infer_volume(teacher.handle, xb, Z3, H3, W3, ob, m.MB_OUT_F32, stream),
                               3, 1, stream, flush)
        t_map = crops_of(ob)
        with torch.cuda.stream(stream):
            ms_s = time_device(lambda: m.mb_infer_volume(student.handle, xb, Z3, H3, W3, ob, m.MB_OUT_F32, stream),
                               3, 1, stream, flush)
        s_map = crops_of(ob)
        teacher_mvox = v3 / (statistics.mean(ms_t) / 1e3) / 1e6
        p8["teacher_bf16_4096x4096x64_mvox_s"] = teacher_mvox
        p8["student_only"] = {"mvox_s": v3 / (statistics.mean(ms_s) / 1e3) / 1e6,
                              "vs_teacher": err_metrics(s_map, t_map, TOL["student"]),
                              "vs_oracle": err_metrics(s_map, c_refs, TOL["student"]),
                              "accuracy_vs_truth": truth_accuracy(s_map, c_truth),
                              "ambiguous_fraction": float(np.mean([((a >= 0.3) & (a <= 0.7)).mean() for a in s_map]))}
        p8["teacher_bf16_crops"] = {"vs_oracle": err_metrics(t_map, c_refs, TOL["bf16"]),
                                    "accuracy_vs_truth": truth_accuracy(t_map, c_truth)}
        p8["oracle_crops_accuracy_vs_truth"] = truth_accuracy(c_refs, c_truth)
        casc = []
        for lo, hi, frac in ((0.3, 0.7, 0.05), (0.3, 0.7, 0.02), (0.3, 0.7, 0.1), (0.1, 0.9, 0.05)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rate = m.mb_infer_cascade(student.handle, teacher.handle, xb, Z3, H3, W3, ob, 256, lo, hi, frac,
                                      stream=stream)
            dt = time.perf_counter() - t0
            c_map = crops_of(ob)
            casc.append({"band": [lo, hi], "tile": 256, "max_frac": frac, "stated_rule": (lo, hi, frac) == (0.3, 0.7, 0.05),
                         "fallback_rate": rate, "mvox_s": v3 / dt / 1e6, "speedup_vs_teacher": v3 / dt / 1e6 / teacher_mvox,
                         "vs_teacher": err_metrics(c_map, t_map, TOL["student"]),
                         "vs_oracle": err_metrics(c_map, c_refs, TOL["student"]),
                         "accuracy_vs_truth": truth_accuracy(c_map, c_truth)})
        p8["cascade"] = casc
        p8["crops"] = crops
        student.close()
        teacher.close()
        paths["cfg8_truth_head_teacher"] = p8
    # ---- cfg5: FastMemb dense form on the cfg1 volume ------------------------------------------------
    if "5" in configs:
        fm_params = synth.init_params(synth.FASTMEMB, synth.FASTMEMB_WEIGHT_SEED)
        rng = np.random.default_rng(synth.BASE_SEED + 5)
        crops = [(int(rng.integers(0, Z)), 2 * int(rng.integers(0, (H - 384) // 2)),
                  2 * int(rng.integers(0, (W - 384) // 2))) for _ in range(3)]
        refs = [oracle.forward_region(synth.FASTMEMB, fm_params, vol[z], y, x0, 384, 384) for z, y, x0 in crops]
        p = {"crops_384": crops}
        for name, prec in (("fp32", m.MB_PREC_FP32), ("bf16", m.MB_PREC_BF16), ("fp16", m.MB_PREC_FP16)):
            tol = TOL["bf16" if name == "fp16" else name]  # FP16 is held to the 16-bit (BF16) bar
            fm = m.Net(synth.FASTMEMB, prec, local, fm_params)
            with torch.cuda.stream(stream):
                ms = time_device(lambda: m.mb_infer_volume(fm.handle, x, Z, H, W, out, m.MB_OUT_F32, stream),
                                 3 if name == "fp32" else args.steps, 1 if name == "fp32" else 3, stream, flush)
            got = [out[z, y:y + 384, x0:x0 + 384].cpu().numpy() for z, y, x0 in crops]
            mv = vox / (statistics.mean(ms) / 1e3) / 1e6
            p[name] = {"mvox_s": mv, "ms": statistics.mean(ms),
                       "tflops": FASTMEMB_FLOP_PER_PX * mv * 1e6 / 1e12,
                       "error": err_metrics(got, refs, tol)}
            # sub-sampled output (factor 2, the pruned fragment tree): every slice's map at even
            # rows and columns; throughput counted in input voxels (and output voxels)
            osub = torch.empty((Z, H // 2, W // 2), dtype=torch.float32, device="cuda")
            with torch.cuda.stream(stream):
                ms = time_device(lambda: m.mb_infer_volume_subsampled(fm.handle, x, Z, H, W, 2, osub, m.MB_OUT_F32,
                                                                      stream),
                                 3 if name == "fp32" else args.steps, 1 if name == "fp32" else 3, stream, flush)
            got = [osub[z, y // 2:(y + 384) // 2, x0 // 2:(x0 + 384) // 2].cpu().numpy() for z, y, x0 in crops]
            p[name + "_subsampled2"] = {
                "input_mvox_s": vox / (statistics.mean(ms) / 1e3) / 1e6,
                "output_mvox_s": vox / 4 / (statistics.mean(ms) / 1e3) / 1e6, "ms": statistics.mean(ms),
                "error": err_metrics(got, [r[::2, ::2] for r in refs], tol)}
            del osub
            fm.close()
        p["bf16"]["speedup_vs_fp32"] = p["bf16"]["mvox_s"] / p["fp32"]["mvox_s"]
        p["fp16"]["speedup_vs_bf16"] = p["fp16"]["mvox_s"] / p["bf16"]["mvox_s"]
        paths["cfg5_fastmemb_1024x1024x32"] = p
    # ---- cfg6: FastMemb_3nm on 2048x2048x8 ----------------------------------------------------------
    if "6" in configs:
        Z6, H6, W6 = 8, 2048, 2048
        f3 = synth.FASTMEMB_3NM
        f3_params = synth.init_params(f3, synth.FASTMEMB_3NM_WEIGHT_SEED, center_head=True)
        vol6 = synth.em_volume(synth.BASE_SEED + 6, Z6, H6, W6)
        x6 = torch.from_numpy(vol6).cuda()
        o6 = torch.empty((Z6, H6, W6), dtype=torch.float32, device="cuda")
        s6 = torch.empty((Z6, H6 // 2, W6 // 2), dtype=torch.float32, device="cuda")
        v6 = Z6 * H6 * W6
        rng = np.random.default_rng(synth.BASE_SEED + 6)
        crops = [(int(rng.integers(0, Z6)), 2 * int(rng.integers(0, (H6 - 256) // 2)),
                  2 * int(rng.integers(0, (W6 - 256) // 2))) for _ in range(2)]
        refs = [oracle.forward_region(f3, f3_params, vol6[z], y, x0, 256, 256) for z, y, x0 in crops]
        p = {"crops_256": crops, "flop_per_px": FASTMEMB3_FLOP_PER_PX}
        for name, prec in (("fp32", m.MB_PREC_FP32), ("bf16", m.MB_PREC_BF16), ("fp16", m.MB_PREC_FP16)):
            tol = TOL["bf16" if name == "fp16" else name]
            fm = m.Net(f3, prec, local, f3_params)
            k, w0 = (2, 1) if name == "fp32" else (args.steps, 3)
            with torch.cuda.stream(stream):
                ms = time_device(lambda: m.mb_infer_volume(fm.handle, x6, Z6, H6, W6, o6, m.MB_OUT_F32, stream),
                                 k, w0, stream, flush)
                ms_s = time_device(lambda: m.mb_infer_volume_subsampled(fm.handle, x6, Z6, H6, W6, 2, s6,
                                                                        m.MB_OUT_F32, stream), k, w0, stream, flush)
            mv = v6 / (statistics.mean(ms) / 1e3) / 1e6
            p[name] = {"mvox_s": mv, "ms": statistics.mean(ms), "tflops": FASTMEMB3_FLOP_PER_PX * mv * 1e6 / 1e12,
                       "error": err_metrics([o6[z, y:y + 256, x0:x0 + 256].cpu().numpy() for z, y, x0 in crops],
                                            refs, tol)}
            p[name + "_subsampled2"] = {
                "input_mvox_s": v6 / (statistics.mean(ms_s) / 1e3) / 1e6,
                "output_mvox_s": v6 / 4 / (statistics.mean(ms_s) / 1e3) / 1e6, "ms": statistics.mean(ms_s),
                "error": err_metrics([s6[z, y // 2:(y + 256) // 2, x0 // 2:(x0 + 256) // 2].cpu().numpy()
                                      for z, y, x0 in crops], [r[::2, ::2] for r in refs], tol)}
            fm.close()
        paths["cfg6_fastmemb3nm_2048x2048x8"] = p
        del x6, o6, s6
    # ---- cfg7: MaskExtend transfer recursion on a 512x512 window ----------------------------------------
    if "7" in configs:
        Z7, H7, W7, N7 = 20, 512, 512, 16
        em7 = synth.em_volume(synth.BASE_SEED + 7, Z7, H7, W7)
        mb7 = synth.membrane_maps(em7)
        sd7 = synth.disk_masks(4, H7, W7, H7 / 2, W7 / 2, H7 / 5, 2.0, -1.0)
        me_params = synth.init_params(synth.MASKEXTEND, synth.MASKEXTEND_WEIGHT_SEED)
        d_em, d_mb, d_sd = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (em7, mb7, sd7))
        # one step's class maps against the oracle on a 128x128 crop with its true context
        y0, x0 = 192, 160
        xp = oracle.maskextend_input(em7, mb7, {-2 + i: sd7[i] for i in range(4)}, 2, 54)
        ref = oracle.run_layers_mc(synth.MASKEXTEND, me_params, xp[:, y0:y0 + 128 + 108, x0:x0 + 128 + 108])
        vox7 = N7 * H7 * W7
        p7, masks_by = {}, {}
        for name, prec in (("fp32", m.MB_PREC_FP32), ("fp16_tcgen05", m.MB_PREC_FP16)):
            me = m.Net(synth.MASKEXTEND, prec, local, me_params)
            masks7 = torch.zeros((N7, H7, W7), dtype=torch.uint8, device="cuda")
            probs7 = torch.zeros((N7, 3, H7, W7), dtype=torch.float32, device="cuda")
            with torch.cuda.stream(stream):
                ms = time_device(lambda: m.mb_mask_extend(me.handle, d_em, d_mb, Z7, H7, W7, d_sd, 2, N7, masks7,
                                                          probs7, stream=stream), 3 if prec == m.MB_PREC_FP32 else 10,
                                 1 if prec == m.MB_PREC_FP32 else 3, stream, flush)
            got = probs7[0, :, y0:y0 + 128, x0:x0 + 128].cpu().numpy()
            mv = vox7 / (statistics.mean(ms) / 1e3) / 1e6
            masks_by[name] = masks7.cpu().numpy()
            p7[name] = {
                "mvox_s": mv, "ms": statistics.mean(ms), "steps_per_s": N7 / (statistics.mean(ms) / 1e3),
                "tflops": MASKEXTEND_FLOP_PER_PX * mv * 1e6 / 1e12,
                "frac_of_sustained_16bit_peak": (MASKEXTEND_FLOP_PER_PX * mv * 1e6 / 1e12 / peaks()[0]["bf16_tflops_sustained"]
                                                 if prec == m.MB_PREC_FP16 else None),
                "mask_fraction": float(masks7.float().mean()),
                "error_step0_crop128": {k: v for k, v in oracle.metrics(got, ref).items()}}
            me.close()
        p7["flop_per_px"] = MASKEXTEND_FLOP_PER_PX
        p7["fp16_vs_fp32_mask_agreement_16_free_steps"] = float((masks_by["fp16_tcgen05"] == masks_by["fp32"]).mean())
        paths["cfg7_maskextend_512x512x16steps"] = p7
    if paths:
        line["paths"] = paths
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    net.close()
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
