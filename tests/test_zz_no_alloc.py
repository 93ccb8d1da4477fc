"""mb_infer_volume_noalloc: the FP32 path for callers that cannot allocate device memory once they
run (fixed memory budget, or no tolerance for the synchronisation of cudaMalloc/cudaFree). Checked
through the C ABI against mb_infer_volume on two calls in a row. Collected last on purpose."""
import numpy as np
import pytest

import synth
from _common import TOL, make_net, teacher_params

pytestmark = pytest.mark.gpu


def test_noalloc_matches_infer_volume_twice():
    import torch
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    net = make_net(synth.TEACHER, m.MB_PREC_FP32, teacher_params())
    lib = m.load()
    for call, (z, h, w) in enumerate([(3, 200, 170), (2, 96, 130)]):
        v = synth.em_volume(5000 + call, z, h, w)
        x = torch.from_numpy(v).cuda()
        ref = torch.empty((z, h, w), dtype=torch.float32, device="cuda")
        got = torch.full((z, h, w), -1.0, dtype=torch.float32, device="cuda")
        m.mb_infer_volume(net.handle, x, z, h, w, ref)
        st = lib.mb_infer_volume_noalloc(net.handle, x.data_ptr(), z, h, w, got.data_ptr(), m.MB_OUT_F32, None)
        assert st == m.MB_OK, m.last_error()
        torch.cuda.synchronize()
        diff = (got - ref).abs().max().item()
        assert diff <= TOL["fp32"]["max_abs"], (call, diff)
    net.close()


def test_noalloc_rejects_what_it_cannot_serve():
    import torch
    from paper_1612_02120_gb300 import membrane as m
    lib = m.load()
    bf = make_net(synth.TEACHER, m.MB_PREC_BF16, teacher_params())
    x = torch.zeros((1, 16, 16), dtype=torch.uint8, device="cuda")
    out = torch.empty((1, 16, 16), dtype=torch.float32, device="cuda")
    assert lib.mb_infer_volume_noalloc(bf.handle, x.data_ptr(), 1, 16, 16, out.data_ptr(), 0, None) == \
        m.MB_ERR_UNSUPPORTED
    bf.close()
    net = make_net(synth.TEACHER, m.MB_PREC_FP32, teacher_params())
    assert lib.mb_infer_volume_noalloc(net.handle, x.data_ptr(), 1, 16, 70000, out.data_ptr(), 0, None) == \
        m.MB_ERR_SHAPE
    assert "maximum" in m.last_error()
    net.close()
