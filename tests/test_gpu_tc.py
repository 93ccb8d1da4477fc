"""Tensor-core fused path (BF16, FP8 E4M3) vs the FP64 oracle at the stated tolerances, plus
the path's invariants (slices independent, region == crop, u8 == rounded float, strips and
row chunks stitch exactly). Calls go through the C ABI."""
import numpy as np
import pytest

import oracle
import synth
from _common import TOL, infer, make_net, teacher_params, within

pytestmark = pytest.mark.gpu

T = synth.TEACHER


@pytest.fixture(scope="module")
def bf16():
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    n = make_net(T, m.MB_PREC_BF16, teacher_params())
    yield n
    n.close()


@pytest.fixture(scope="module")
def fp8():
    import torch
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    n = make_net(T, m.MB_PREC_FP8, teacher_params())
    cal = torch.from_numpy(synth.em_volume(synth.BASE_SEED + 3, 4, 256, 256)).cuda()
    amax = np.zeros(64, dtype=np.float32)
    m.mb_calibrate_fp8(n.handle, cal, 4, 256, 256, amax)
    n.amax = amax
    n.cal = cal.cpu().numpy()
    yield n
    n.close()


def test_bf16_single_slice_256(bf16):
    s = synth.em_slice(synth.slice_seed(synth.BASE_SEED, 0, 0), 256, 256)
    p = infer(bf16, s[None])[0]
    met = oracle.metrics(p, oracle.forward_region(T, teacher_params(), s))
    assert within(met, TOL["bf16"]), met


@pytest.mark.parametrize("shape", [(1, 8, 8), (2, 16, 17), (1, 37, 130), (2, 70, 250), (1, 129, 9)])
def test_bf16_odd_shapes(bf16, shape):
    z, h, w = shape
    v = synth.em_volume(2000 + h * w, z, h, w)
    p = infer(bf16, v)
    for zi in range(z):
        met = oracle.metrics(p[zi], oracle.forward_region(T, teacher_params(), v[zi]))
        assert met["max_abs"] <= TOL["bf16"]["max_abs"], (shape, zi, met)


def test_bf16_slices_independent_and_deterministic(bf16):
    v = synth.em_volume(91, 3, 96, 130)
    a = infer(bf16, v)
    np.testing.assert_array_equal(a, infer(bf16, v))
    for zi in range(3):
        np.testing.assert_array_equal(a[zi], infer(bf16, v[zi:zi + 1])[0])


def test_bf16_region_equals_crop(bf16):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    v = synth.em_volume(92, 2, 150, 260)
    full = infer(bf16, v)
    x = torch.from_numpy(v).cuda()
    out = torch.empty((2, 61, 133), dtype=torch.float32, device="cuda")
    m.mb_infer_region(bf16.handle, x, 2, 150, 260, 40, 100, 61, 133, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), full[:, 40:101, 100:233])


def test_bf16_u8_output(bf16):
    v = synth.em_volume(93, 1, 64, 200)
    pf = infer(bf16, v, 0)
    pq = infer(bf16, v, 1)
    q = np.minimum(255, np.floor(np.float32(255.0) * pf + np.float32(0.5))).astype(np.uint8)
    np.testing.assert_array_equal(pq, q)


def test_bf16_row_chunking_does_not_change_results(bf16):
    """Items of different row counts stitch to the same map (each output row is computed with its
    true context)."""
    from paper_1612_02120_gb300 import membrane as m
    v = synth.em_volume(94, 1, 300, 140)
    a = infer(bf16, v)
    m.mb_autotune  # the tuned rows-per-item is exercised in test_gpu_batch
    ref = oracle.forward_region(T, teacher_params(), v[0])
    assert oracle.metrics(a[0], ref)["max_abs"] <= TOL["bf16"]["max_abs"]


def test_bf16_full_size_sampled(bf16):
    """1024x1024x32 in the bench's launch configuration: 2 seeded slices in full vs the oracle,
    plus single pixels at strip seams, borders and corners of every slice via the patch form."""
    v = synth.em_volume(synth.BASE_SEED + 1, 32, 1024, 1024)
    p = infer(bf16, v)
    rng = np.random.default_rng(5)
    params = teacher_params()
    for zi in rng.choice(32, size=2, replace=False):
        met = oracle.metrics(p[zi], oracle.forward_region(T, params, v[zi]))
        assert within(met, TOL["bf16"]), (zi, met)
    pts = [(0, 0), (0, 1023), (1023, 0), (1023, 1023), (511, 117), (511, 118), (3, 236), (1020, 944)]
    for zi in range(0, 32, 5):
        for (i, j) in pts:
            ref = oracle.patch_pixel(T, params, v[zi], i, j)
            assert abs(p[zi, i, j] - ref) <= TOL["bf16"]["max_abs"], (zi, i, j)


def test_fp8_calibration_amax_matches_oracle(fp8):
    params = teacher_params()
    ref = np.max([oracle.maxfilter_amax(T, params, s) for s in fp8.cal], axis=0).reshape(-1)
    np.testing.assert_allclose(fp8.amax, ref, rtol=1e-5, atol=1e-6)


def test_fp8_single_slice_256(fp8):
    s = synth.em_slice(synth.slice_seed(synth.BASE_SEED, 0, 0), 256, 256)
    p = infer(fp8, s[None])[0]
    met = oracle.metrics(p, oracle.forward_region(T, teacher_params(), s))
    assert within(met, TOL["fp8"]), met


def test_fp8_uncalibrated_is_not_ready():
    import ctypes
    import torch
    from paper_1612_02120_gb300 import membrane as m
    n = make_net(T, m.MB_PREC_FP8, teacher_params())
    x = torch.zeros((1, 16, 16), dtype=torch.uint8, device="cuda")
    out = torch.empty((1, 16, 16), dtype=torch.float32, device="cuda")
    assert m.load().mb_infer_volume(n.handle, x.data_ptr(), 1, 16, 16, out.data_ptr(), 0, None) == m.MB_ERR_NOT_READY
    n.close()


@pytest.mark.parametrize("z", [30, 23, 15])
def test_host_streaming_over_several_slabs_equals_device_path(z):
    """1024x1024xz from pinned host buffers streams in slabs of at most 8 slices: for 30 slices
    4, 8, 8, 6, 4 (half-size first and last slabs, a ragged one before the last), for 23 4, 8, 7, 4,
    for 15 8, 7 (too short to halve the ends); slabs alternate between two buffers and, for this
    tensor-core net, two compute streams. The maps equal the device-resident call bitwise."""
    import torch
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    net = make_net(T, m.MB_PREC_BF16, teacher_params())
    v = synth.em_volume(5100, z, 1024, 1024)
    dev = infer(net, v)
    pin_in = torch.from_numpy(v).pin_memory()
    pin_out = torch.empty((z, 1024, 1024), dtype=torch.float32).pin_memory()
    m.mb_set_host_io(net.handle, m.MB_HOST_IO_SLABS)  # pinned buffers would otherwise be accessed directly
    for _ in range(2):  # the second call reuses the net's slab buffers, streams and events
        pin_out.fill_(-1.0)
        m.mb_infer_volume(net.handle, pin_in, z, 1024, 1024, pin_out)
        np.testing.assert_array_equal(pin_out.numpy(), dev)
    m.mb_set_host_io(net.handle, m.MB_HOST_IO_AUTO)
    pin_out.fill_(-1.0)
    m.mb_infer_volume(net.handle, pin_in, z, 1024, 1024, pin_out)
    np.testing.assert_array_equal(pin_out.numpy(), dev)
    net.close()
