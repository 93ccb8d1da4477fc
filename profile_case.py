"""Bench helper, not part of the library: small, fixed inference cases for profilers (ncu
captures of one kernel). `reps` launches of one path on a z x h x w synthetic volume (the
generator of `synth`), so a capture of one kernel stays a few hundred MB on the device.

    python profile_case.py --prec bf16 --z 4 --h 1024 --w 1024 --reps 3 [--rows 1024 --stages 6]
    python profile_case.py --net fastmemb --prec bf16 --z 4 --reps 3
    python profile_case.py --net maskextend --prec fp16 --z 4 --h 512 --w 512
      (MaskExtend: `z` transfer steps on an h x w window per rep)
    python profile_case.py --net student-train --z 64 --h 512 --w 512 --reps 4
      (student training: `reps` optimiser steps, batch 32, on z slices with FP32 teacher targets)
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--net", default="teacher", choices=["teacher", "fastmemb", "maskextend", "student-train"])
    ap.add_argument("--prec", default="bf16", choices=["fp32", "bf16", "fp8", "fp16", "student"])
    ap.add_argument("--z", type=int, default=4)
    ap.add_argument("--h", type=int, default=1024)
    ap.add_argument("--w", type=int, default=1024)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--rows", type=int, default=0, help="teacher: rows per work item (mb_set_tuning); 0 keeps the default")
    ap.add_argument("--stages", type=int, default=0, help="teacher: A-ring depth (mb_set_tuning); 0 keeps the default")
    a = ap.parse_args()
    import torch

    import synth
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    if a.net == "student-train":
        v = torch.from_numpy(synth.em_volume(synth.BASE_SEED + 4, a.z, a.h, a.w)).cuda()
        tgt = torch.empty((a.z, a.h, a.w), dtype=torch.float32, device="cuda")
        with m.Net(synth.TEACHER, m.MB_PREC_FP32, 0, synth.init_params(synth.TEACHER, synth.TEACHER_WEIGHT_SEED)) as t:
            m.mb_infer_volume(t.handle, v, a.z, a.h, a.w, tgt)
        sp = synth.init_params(synth.STUDENT, synth.STUDENT_WEIGHT_SEED, bias_std=0.0)
        with m.Net(synth.STUDENT, m.MB_PREC_BF16, 0, sp) as st:
            m.mb_student_train(st.handle, v, tgt, a.z, a.h, a.w,
                               m.train_cfg(batch=32, steps=a.reps, lr=1e-3, seed=synth.BASE_SEED + 4))
        torch.cuda.synchronize()
        print(f"ok student-train {a.reps} steps, batch 32 of {a.z}x{a.h}x{a.w}")
        return
    if a.net == "maskextend":
        em = synth.em_volume(synth.BASE_SEED + 7, a.z + 4, a.h, a.w)
        d = [torch.from_numpy(arr).cuda() for arr in
             (em, synth.membrane_maps(em), synth.disk_masks(4, a.h, a.w, a.h / 2, a.w / 2, a.h / 5, 2.0, -1.0))]
        prec = {"fp32": m.MB_PREC_FP32, "fp16": m.MB_PREC_FP16}[a.prec]
        net = m.Net(synth.MASKEXTEND, prec, 0, synth.init_params(synth.MASKEXTEND, synth.MASKEXTEND_WEIGHT_SEED))
        masks = torch.zeros((a.z, a.h, a.w), dtype=torch.uint8, device="cuda")
        for _ in range(a.reps):
            m.mb_mask_extend(net.handle, d[0], d[1], a.z + 4, a.h, a.w, d[2], 2, a.z, masks, None)
        torch.cuda.synchronize()
        print(f"ok maskextend {a.prec} {a.z} steps of {a.h}x{a.w} mask fraction {float(masks.float().mean()):.6f}")
        net.close()
        return
    v = synth.em_volume(synth.BASE_SEED + 1, a.z, a.h, a.w)
    x = torch.from_numpy(v).cuda()
    out = torch.empty((a.z, a.h, a.w), dtype=torch.float32, device="cuda")
    if a.net == "fastmemb":
        prec = {"fp32": m.MB_PREC_FP32, "bf16": m.MB_PREC_BF16, "fp16": m.MB_PREC_FP16}[a.prec]
        net = m.Net(synth.FASTMEMB, prec, 0, synth.init_params(synth.FASTMEMB, synth.FASTMEMB_WEIGHT_SEED))
    elif a.prec == "student":
        net = m.Net(synth.STUDENT, m.MB_PREC_BF16, 0, synth.init_params(synth.STUDENT, synth.STUDENT_WEIGHT_SEED))
    else:
        prec = {"fp32": m.MB_PREC_FP32, "bf16": m.MB_PREC_BF16, "fp8": m.MB_PREC_FP8}[a.prec]
        net = m.Net(synth.TEACHER, prec, 0, synth.init_params(synth.TEACHER, synth.TEACHER_WEIGHT_SEED))
        if prec == m.MB_PREC_FP8:
            m.mb_calibrate_fp8(net.handle, x[: min(4, a.z)], min(4, a.z), a.h, a.w)
        if a.stages and prec != m.MB_PREC_FP32:
            m.mb_set_tuning(net.handle, a.rows if prec == m.MB_PREC_BF16 else 0, a.stages)
    for _ in range(a.reps):
        m.mb_infer_volume(net.handle, x, a.z, a.h, a.w, out)
    torch.cuda.synchronize()
    print(f"ok {a.net} {a.prec} {a.z}x{a.h}x{a.w} mean p {float(out.mean()):.6f}")
    net.close()


if __name__ == "__main__":
    main()
