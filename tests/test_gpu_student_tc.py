"""BF16 student inference on the tensor cores (the fused kernel of student_tc.cu) through the C ABI:
parity with the FP64 oracle (BF16-rounded weights) at the BF16 bar over slice shapes that span
strips, ragged edges and the minimum size; regions with their true context; uint8 output; host
buffers; batches; a volume against its slices one by one; a sampled check at a large size; a
timed-out device wait."""
import numpy as np
import pytest

import oracle
import synth
from _common import TOL, infer, make_net, student_params, within

pytestmark = pytest.mark.gpu

S = synth.STUDENT


def bf16_round(a):
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def net():
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    n = make_net(S, m.MB_PREC_BF16, student_params())
    yield n
    n.close()


@pytest.mark.parametrize("shape", [(1, 8, 8), (2, 70, 45), (1, 300, 530), (1, 1000, 9), (3, 129, 257)])
def test_bf16_student_matches_oracle(net, shape):
    """Binarised agreement is a statistic over the map: asserted on maps of at least 4096 pixels
    (on 8x8 one pixel within the error of the threshold is already 1.6 %)."""
    v = synth.em_volume(7100 + shape[1], *shape)
    out = infer(net, v)
    pref = bf16_round(student_params())
    tol = dict(TOL["bf16"])
    if shape[1] * shape[2] < 4096:
        tol.pop("agreement")
    for zi in range(shape[0]):
        met = oracle.metrics(out[zi], oracle.forward_region(S, pref, v[zi]))
        assert within(met, tol), met


def test_region_equals_crop_of_full_map(net):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    v = synth.em_volume(7200, 2, 150, 300)
    full = infer(net, v)
    x = torch.from_numpy(v).cuda()
    for y0, x0, r, c in ((0, 0, 40, 50), (37, 131, 100, 169), (149, 299, 1, 1)):
        out = torch.empty((2, r, c), dtype=torch.float32, device="cuda")
        m.mb_infer_region(net.handle, x, 2, 150, 300, y0, x0, r, c, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), full[:, y0:y0 + r, x0:x0 + c])


def test_u8_host_and_batch_paths(net):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    v = synth.em_volume(7300, 3, 90, 140)
    pf = infer(net, v)
    pq = infer(net, v, 1)
    np.testing.assert_array_equal(pq, np.minimum(255, np.floor(np.float32(255.0) * pf + np.float32(0.5))).astype(np.uint8))
    host = np.empty((3, 90, 140), dtype=np.float32)
    m.mb_infer_volume(net.handle, np.ascontiguousarray(v), 3, 90, 140, host)
    np.testing.assert_array_equal(host, pf)
    x = torch.from_numpy(v).cuda()
    outs = [torch.empty((1, 90, 140), dtype=torch.float32, device="cuda") for _ in range(3)]
    blocks = [(x[i:i + 1], 1, 90, 140, 140, 90 * 140, outs[i], 140, 90 * 140) for i in range(3)]
    m.mb_infer_batch(net.handle, blocks)
    torch.cuda.synchronize()
    for i in range(3):
        np.testing.assert_array_equal(outs[i].cpu().numpy()[0], pf[i])


def test_volume_equals_slice_by_slice(net):
    """A many-slice launch walks every CTA's rings (operand, accumulator and staged-row slots and
    their phases) through many wraps and item boundaries at other offsets than one-slice launches
    do; the maps must not depend on where a row falls in them."""
    v = synth.em_volume(7350, 7, 333, 517)
    full = infer(net, v)
    for zi in range(7):
        np.testing.assert_array_equal(infer(net, v[zi:zi + 1])[0], full[zi])


def test_sampled_crops_at_a_large_size(net):
    v = synth.em_volume(7400, 2, 2048, 2048)
    out = infer(net, v)
    pref = bf16_round(student_params())
    for zi, y0, x0 in ((0, 0, 0), (1, 1500, 777), (0, 1920, 1920)):
        ref = oracle.forward_region(S, pref, v[zi], y0, x0, 128, 128)
        met = oracle.metrics(out[zi, y0:y0 + 128, x0:x0 + 128], ref)
        assert within(met, TOL["bf16"]), met


def test_timed_out_device_wait_is_reported_and_context_survives(net, monkeypatch):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    lib = m.load()
    v = synth.em_volume(7500, 1, 64, 80)
    ref = infer(net, v)
    x = torch.from_numpy(v).cuda()
    out = torch.zeros((1, 64, 80), dtype=torch.float32, device="cuda")
    monkeypatch.setenv("MB_FAULT_STALL", "1")
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), 1, 64, 80, out.data_ptr(), 0, None) == m.MB_OK
    torch.cuda.synchronize()
    monkeypatch.delenv("MB_FAULT_STALL")
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), 1, 64, 80, out.data_ptr(), 0, None) == m.MB_ERR_TIMEOUT
    assert "wait limit" in m.last_error()
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), 1, 64, 80, out.data_ptr(), 0, None) == m.MB_OK
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
