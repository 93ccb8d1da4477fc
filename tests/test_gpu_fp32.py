"""FP32 CUDA-core path vs the FP64 oracle, element by element (max-abs <= 1e-5), plus the
path's invariants. Calls go through the C ABI."""
import numpy as np
import pytest

import oracle
import synth
from _common import TOL, infer, make_net, teacher_params, within

pytestmark = pytest.mark.gpu

T = synth.TEACHER


@pytest.fixture(scope="module")
def net():
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    n = make_net(T, m.MB_PREC_FP32, teacher_params())
    yield n
    n.close()


def test_single_slice_256_matches_oracle(net):
    """One 256x256 slice of the generator (120 cells), full map."""
    s = synth.em_slice(synth.slice_seed(synth.BASE_SEED, 0, 0), 256, 256)
    p = infer(net, s[None])[0]
    ref = oracle.forward_region(T, teacher_params(), s)
    met = oracle.metrics(p, ref)
    assert within(met, TOL["fp32"]), met


@pytest.mark.parametrize("shape", [(1, 8, 8), (2, 16, 17), (1, 37, 130), (3, 70, 33), (1, 9, 300)])
def test_odd_shapes_match_oracle(net, shape):
    z, h, w = shape
    v = synth.em_volume(1000 + h * w, z, h, w)
    p = infer(net, v)
    for zi in range(z):
        ref = oracle.forward_region(T, teacher_params(), v[zi])
        met = oracle.metrics(p[zi], ref)
        assert met["max_abs"] <= TOL["fp32"]["max_abs"], (shape, zi, met)


def test_u8_output_is_rounded_float_output(net):
    v = synth.em_volume(77, 2, 64, 96)
    pf = infer(net, v, 0)
    pq = infer(net, v, 1)
    q = np.minimum(255, np.floor(np.float32(255.0) * pf + np.float32(0.5))).astype(np.uint8)
    np.testing.assert_array_equal(pq, q)
    ref = oracle.forward_region(T, teacher_params(), v[0])
    assert np.abs(pq[0].astype(np.int32) - np.minimum(255, np.floor(255 * ref + 0.5))).max() <= 1


def test_slices_are_independent(net):
    v = synth.em_volume(78, 4, 48, 40)
    all_ = infer(net, v)
    for zi in range(4):
        np.testing.assert_array_equal(all_[zi], infer(net, v[zi:zi + 1])[0])


def test_region_equals_volume_crop(net):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    v = synth.em_volume(79, 2, 100, 90)
    full = infer(net, v)
    x = torch.from_numpy(v).cuda()
    out = torch.empty((2, 31, 45), dtype=torch.float32, device="cuda")
    m.mb_infer_region(net.handle, x, 2, 100, 90, 60, 3, 31, 45, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), full[:, 60:91, 3:48])


def test_host_pointers_stream_in_slabs_and_match_device_path(net):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    v = synth.em_volume(80, 5, 64, 72)
    dev = infer(net, v)
    pin_in = torch.from_numpy(v).pin_memory()
    pin_out = torch.empty((5, 64, 72), dtype=torch.float32).pin_memory()
    for mode in (m.MB_HOST_IO_SLABS, m.MB_HOST_IO_AUTO):
        m.mb_set_host_io(net.handle, mode)
        pin_out.fill_(-1.0)
        m.mb_infer_volume(net.handle, pin_in, 5, 64, 72, pin_out)
        np.testing.assert_array_equal(pin_out.numpy(), dev)
    pageable_out = np.empty((5, 64, 72), dtype=np.float32)
    m.mb_infer_volume(net.handle, np.ascontiguousarray(v), 5, 64, 72, pageable_out)
    np.testing.assert_array_equal(pageable_out, dev)


def test_translation_equivariance_on_gpu(net):
    big = synth.em_slice(81, 80, 80)
    dy, dx = 6, 11
    a = infer(net, big[None, 0:60, 0:60].copy())[0]
    b = infer(net, big[None, dy:dy + 60, dx:dx + 60].copy())[0]
    np.testing.assert_array_equal(a[dy + 7:60 - 7, dx + 7:60 - 7], b[7:60 - 7 - dy, 7:60 - 7 - dx])


def test_error_codes(net):
    import ctypes
    import torch
    from paper_1612_02120_gb300 import membrane as m
    lib = m.load()
    x = torch.zeros((1, 7, 64), dtype=torch.uint8, device="cuda")
    out = torch.empty((1, 7, 64), dtype=torch.float32, device="cuda")
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), 1, 7, 64, out.data_ptr(), 0, None) == m.MB_ERR_SHAPE
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), 1, 64, 7, out.data_ptr(), 0, None) == m.MB_ERR_SHAPE
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), 1, 8, 8, out.data_ptr(), 5, None) == m.MB_ERR_INVALID_ARG
    host = np.zeros((1, 8, 8), dtype=np.float32)
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), 1, 8, 8, host.ctypes.data, 0, None) == m.MB_ERR_INVALID_ARG
    fresh = m.mb_net_create(T, m.MB_PREC_FP32, 0)
    assert lib.mb_infer_volume(fresh, x.data_ptr(), 1, 8, 8, out.data_ptr(), 0, None) == m.MB_ERR_NOT_READY
    short = np.zeros(10, dtype=np.float32)
    assert lib.mb_load_weights(fresh, short.ctypes.data, 10) == m.MB_ERR_INVALID_ARG
    nan = teacher_params().copy()
    nan[5] = np.nan
    assert lib.mb_load_weights(fresh, nan.ctypes.data, nan.size) == m.MB_ERR_INVALID_ARG
    m.mb_net_destroy(fresh)
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), 0, 8, 8, out.data_ptr(), 0, None) == m.MB_OK


def test_injected_allocation_failure_reports_oom(monkeypatch):
    from paper_1612_02120_gb300 import membrane as m
    monkeypatch.setenv("MB_FAULT_OOM", "1")
    with pytest.raises(m.MembraneError) as e:
        m.mb_net_create(T, m.MB_PREC_FP32, 0)
    assert e.value.status == m.MB_ERR_OOM
