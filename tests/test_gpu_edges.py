"""Edge cases through the C ABI against the FP64 oracle: extreme aspect ratios at the minimum
slice sizes (8 for the teacher, 27 for FastMemb, 55 for MaskExtend), and the maximum-size and
empty-input rules, which are decided before any device work."""
import numpy as np
import pytest

import oracle
import synth
from _common import TOL, infer, make_net, teacher_params, within

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(1, 8, 9001), (1, 2999, 8)])
def test_teacher_bf16_thin_slices(shape):
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    net = make_net(synth.TEACHER, m.MB_PREC_BF16, teacher_params())
    v = synth.em_volume(6100 + shape[1], *shape)
    met = oracle.metrics(infer(net, v)[0], oracle.forward_region(synth.TEACHER, teacher_params(), v[0]))
    net.close()
    assert within(met, TOL["bf16"]), met


@pytest.mark.parametrize("shape", [(1, 27, 3001), (1, 2001, 27)])
def test_fastmemb_thin_slices(shape):
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    prm = synth.init_params(synth.FASTMEMB, synth.FASTMEMB_WEIGHT_SEED)
    v = synth.em_volume(6200 + shape[1], *shape)
    ref = oracle.forward_region(synth.FASTMEMB, prm, v[0])
    for prec, tol in ((m.MB_PREC_FP32, TOL["fp32"]), (m.MB_PREC_BF16, TOL["bf16"])):
        net = make_net(synth.FASTMEMB, prec, prm)
        met = oracle.metrics(infer(net, v)[0], ref)
        net.close()
        assert within(met, tol), (prec, met)


def test_maskextend_minimum_section():
    import torch
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    prm = synth.init_params(synth.MASKEXTEND, synth.MASKEXTEND_WEIGHT_SEED)
    em = synth.em_volume(6300, 5, 55, 55)
    memb = synth.membrane_maps(em)
    seeds = synth.disk_masks(4, 55, 55, 27, 27, 12)
    net = make_net(synth.MASKEXTEND, m.MB_PREC_FP32, prm)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (em, memb, seeds)]
    masks = torch.zeros((1, 55, 55), dtype=torch.uint8, device="cuda")
    probs = torch.zeros((1, 3, 55, 55), dtype=torch.float32, device="cuda")
    m.mb_mask_extend(net.handle, d[0], d[1], 5, 55, 55, d[2], 2, 1, masks, probs)
    torch.cuda.synchronize()
    net.close()
    _, ref = oracle.mask_extend(synth.MASKEXTEND, prm, em, memb, seeds, 2, 1)
    assert oracle.metrics(probs.cpu().numpy(), ref)["max_abs"] <= TOL["fp32"]["max_abs"]


def test_size_rules_are_decided_before_device_work():
    import torch
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    lib = m.load()
    net = make_net(synth.TEACHER, m.MB_PREC_BF16, teacher_params())
    x = torch.zeros(64, dtype=torch.uint8, device="cuda")
    y = torch.zeros(64, dtype=torch.float32, device="cuda")
    big = (1 << 20) + 1
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), 1, 8, big, y.data_ptr(), 0, None) == m.MB_ERR_SHAPE
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), 1, big, 8, y.data_ptr(), 0, None) == m.MB_ERR_SHAPE
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), -1, 8, 8, y.data_ptr(), 0, None) == m.MB_ERR_INVALID_ARG
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), 0, 8, 8, y.data_ptr(), 0, None) == m.MB_OK
    assert lib.mb_infer_batch(net.handle, None, 0, 0, None) == m.MB_OK
    assert lib.mb_infer_region(net.handle, x.data_ptr(), 1, 8, 8, 0, 0, 0, 0, y.data_ptr(), 0, None) == m.MB_OK
    net.close()
