"""Helpers shared by the GPU tests: nets with seeded weights, inference through the C ABI, and the
stated error tolerances (fixed before the first measurement, never loosened)."""
import numpy as np

import synth

TOL = {
    # max-abs / mean-abs vs the FP64 oracle, and binarised agreement at p = 0.5
    "fp32": {"max_abs": 1e-5, "agreement": 0.995},
    "bf16": {"max_abs": 3e-2, "mean_abs": 2e-3, "agreement": 0.995},
    "fp8": {"max_abs": 1e-1, "mean_abs": 1e-2, "agreement": 0.995},
    # MaskExtend on the tensor cores (FP16 operands): held to the 16-bit (BF16) bar
    "fp16": {"max_abs": 3e-2, "mean_abs": 2e-3},
    "student": {"mean_abs": 3e-2, "agreement": 0.995},
}


def teacher_params():
    return synth.init_params(synth.TEACHER, synth.TEACHER_WEIGHT_SEED)


def truth_head_teacher_params():
    """The second teacher workload: the stand-in teacher with its head fitted to the generator's
    membrane truth (tests/golden/truth_head.json, written by fit_truth_head.py from the oracle)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "truth_head.json")) as f:
        fx = json.load(f)
    p = teacher_params().copy()
    p[-33:-1] = np.asarray(fx["head_w"], dtype=np.float32)
    p[-1] = np.float32(fx["head_b"])
    return p


def student_params():
    return synth.init_params(synth.STUDENT, synth.STUDENT_WEIGHT_SEED, bias_std=0.0, centred_input=True)


def make_net(layers, prec, params):
    from paper_1612_02120_gb300 import membrane as m
    return m.Net(layers, prec, 0, params)


def infer(net, vol_u8, out_type=0, stream=None):
    """vol_u8: numpy [z][h][w] uint8 -> numpy map (float32 or uint8) via device buffers."""
    import torch
    from paper_1612_02120_gb300 import membrane as m
    x = torch.from_numpy(np.ascontiguousarray(vol_u8)).cuda()
    z, h, w = vol_u8.shape
    out = torch.empty((z, h, w), dtype=torch.float32 if out_type == 0 else torch.uint8, device="cuda")
    m.mb_infer_volume(net.handle, x, z, h, w, out, out_type, stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def within(metrics, tol):
    ok = True
    for k, v in tol.items():
        if k == "agreement":
            ok &= metrics[k] >= v
        else:
            ok &= metrics[k] <= v
    return ok
