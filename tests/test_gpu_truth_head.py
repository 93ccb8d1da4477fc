"""The second teacher workload: the stand-in teacher with its head fitted to the synthetic
generator's membrane truth (tests/golden/truth_head.json), a map that straddles 0.5 like a trained
membrane classifier's. Through the C ABI, against the FP64 oracle and the generator's truth.

The fitted head is steep and ill-conditioned: kappa = |b| + sum_c |w_c| h_c is about 70-83 per pixel
(the stand-in head: about 2.4), so every rounding error inside the network reaches the logit
amplified ~30x. The FP32 check is therefore the per-pixel forward-error bound
    |p_gpu - p_64| <= 1e-5 + p (1 - p) kappa 2^-17
(a relative logit error of 64 FP32 ulps; the stand-in head's FP32 path measures about 8), not the
plain 1e-5 of the stand-in. BF16 and FP8 are checked on what they preserve: the task accuracy
against the generator's truth."""
import numpy as np
import pytest

import oracle
import synth
from _common import TOL, infer, make_net, truth_head_teacher_params

pytestmark = pytest.mark.gpu

T = synth.TEACHER


@pytest.fixture(scope="module")
def data():
    from paper_1612_02120_gb300 import build
    build.build()
    base = synth.BASE_SEED + 24
    sl = [synth.em_slice_truth(synth.slice_seed(base, 0, i), 256, 300) for i in range(2)]
    vol = np.stack([s for s, _ in sl])
    truth = np.stack([t for _, t in sl])
    p = truth_head_teacher_params()
    ref = np.stack([oracle.forward_region(T, p, s) for s in vol])
    w, b = p[-33:-1].astype(np.float64), float(p[-1])
    kappa = np.stack([abs(b) + np.einsum("c,chw->hw", np.abs(w), oracle.features(T, p, s)) for s in vol])
    return vol, truth, p, ref, kappa


def accuracy(pm, truth):
    return float(((pm >= 0.5) == (truth > 0)).mean())


def test_fp32_within_the_conditioned_bound(data):
    from paper_1612_02120_gb300 import membrane as m
    vol, truth, p, ref, kappa = data
    net = make_net(T, m.MB_PREC_FP32, p)
    got = infer(net, vol).astype(np.float64)
    bound = 1e-5 + ref * (1 - ref) * kappa * 2.0 ** -17
    err = np.abs(got - ref)
    assert (err <= bound).all(), (err.max(), float((err / bound).max()))
    assert float(np.median(kappa)) > 20       # the workload is the ill-conditioned one
    assert accuracy(got, truth) == accuracy(ref, truth)
    net.close()


def test_bf16_keeps_the_task_accuracy(data):
    from paper_1612_02120_gb300 import membrane as m
    vol, truth, p, ref, _ = data
    net = make_net(T, m.MB_PREC_BF16, p)
    got = infer(net, vol)
    met = oracle.metrics(got, ref)
    assert met["mean_abs"] <= TOL["bf16"]["mean_abs"] and met["agreement"] >= 0.995, met
    assert abs(accuracy(got, truth) - accuracy(ref, truth)) <= 0.002
    net.close()


def test_fp8_task_accuracy_cost_is_bounded(data):
    """FP8 E4M3 misses the stated FP8 error bars on this head (recorded by the bench); what it
    costs in accuracy against the truth stays within 1.5 percentage points."""
    import torch
    from paper_1612_02120_gb300 import membrane as m
    vol, truth, p, ref, _ = data
    net = make_net(T, m.MB_PREC_FP8, p)
    cal = torch.from_numpy(synth.em_volume(synth.BASE_SEED + 3, 4, 256, 256)).cuda()
    m.mb_calibrate_fp8(net.handle, cal, 4, 256, 256)
    got = infer(net, vol)
    assert accuracy(ref, truth) - accuracy(got, truth) <= 0.015, (accuracy(ref, truth), accuracy(got, truth))
    assert oracle.metrics(got, ref)["agreement"] >= 0.95
    net.close()
