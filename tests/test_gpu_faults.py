"""Failure detection without a GPU fault: a device-side wait that runs out (the input loader is
told to withhold its arrivals, a flag nothing else sets) ends the kernel cleanly, the host reads
MB_ERR_TIMEOUT, and the context stays usable. Injection is host-side (environment)."""
import numpy as np
import pytest

import synth
from _common import infer, make_net, teacher_params

pytestmark = pytest.mark.gpu


def test_timed_out_device_wait_is_reported_and_context_survives(monkeypatch):
    import time
    import torch
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    net = make_net(synth.TEACHER, m.MB_PREC_BF16, teacher_params())
    lib = m.load()
    v = synth.em_volume(6001, 2, 64, 96)
    ref = infer(net, v)
    x = torch.from_numpy(v).cuda()
    out = torch.zeros((2, 64, 96), dtype=torch.float32, device="cuda")
    monkeypatch.setenv("MB_FAULT_STALL", "1")
    t0 = time.perf_counter()
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), 2, 64, 96, out.data_ptr(), 0, None) == m.MB_OK
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 30.0
    monkeypatch.delenv("MB_FAULT_STALL")
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), 2, 64, 96, out.data_ptr(), 0, None) == m.MB_ERR_TIMEOUT
    assert "wait limit" in m.last_error()
    # the error was consumed; the context and the net still work
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), 2, 64, 96, out.data_ptr(), 0, None) == m.MB_OK
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    net.close()
