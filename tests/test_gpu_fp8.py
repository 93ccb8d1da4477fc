"""FP8 E4M3 teacher (layers 2-3 in E4M3 with per-output-channel weight scales and calibrated
activation scales, FP32 accumulation, FP32 layer 1 and head) against the FP64 oracle at the
stated FP8 tolerances, where its work split has seams. The FP8 kernel cuts a launch's strip-rows,
in (block, slice, strip, row) order, into one equal contiguous range per CTA, so ranges start and
end mid-strip, mid-slice and mid-block; every output row must still be computed with its full
context. Through the C ABI."""
import numpy as np
import pytest

import oracle
import synth
from _common import TOL, infer, make_net, teacher_params, within

pytestmark = pytest.mark.gpu

T = synth.TEACHER
STRIP = 118        # valid output columns per 128-pixel strip of the tensor-core kernel


def calibrated(vol_u8):
    import torch
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    n = make_net(T, m.MB_PREC_FP8, teacher_params())
    z, h, w = vol_u8.shape
    cal = torch.from_numpy(np.ascontiguousarray(vol_u8[:4])).cuda()
    m.mb_calibrate_fp8(n.handle, cal, min(4, z), h, w)
    return n


@pytest.fixture(scope="module")
def fp8():
    n = calibrated(synth.em_volume(synth.BASE_SEED + 3, 4, 256, 256))
    yield n
    n.close()


def check_fp8(p, ref, what, agreement=True):
    met = oracle.metrics(p, ref)
    tol = dict(TOL["fp8"])
    if not agreement or ref.size < 4096:  # agreement is a statistic over a map of >= 4096 pixels
        tol.pop("agreement")
    assert within(met, tol), (what, met)


@pytest.mark.parametrize("shape", [(1, 8, 8), (2, 16, 17), (1, 37, 130), (2, 70, 250), (1, 129, 9), (3, 200, 300)])
def test_fp8_odd_shapes_and_multi_slice(fp8, shape):
    z, h, w = shape
    v = synth.em_volume(6000 + h * w, z, h, w)
    p = infer(fp8, v)
    for zi in range(z):
        check_fp8(p[zi], oracle.forward_region(T, teacher_params(), v[zi]), (shape, zi))


def test_fp8_slices_independent_of_the_range_split(fp8):
    """A slice computed inside a volume (its rows split over the CTAs' ranges at other offsets)
    equals the same slice computed alone, bitwise."""
    v = synth.em_volume(6101, 5, 130, 390)
    a = infer(fp8, v)
    np.testing.assert_array_equal(a, infer(fp8, v))
    for zi in range(5):
        np.testing.assert_array_equal(a[zi], infer(fp8, v[zi:zi + 1])[0])


def test_fp8_u8_output_is_rounded_float(fp8):
    v = synth.em_volume(6102, 2, 64, 200)
    pf = infer(fp8, v, 0)
    pq = infer(fp8, v, 1)
    q = np.minimum(255, np.floor(np.float32(255.0) * pf + np.float32(0.5))).astype(np.uint8)
    np.testing.assert_array_equal(pq, q)


def range_seams(z, h, w, n_sms):
    """(slice, row, strip) at which a CTA's range of the FP8 even split begins, for a launch of one
    z x h x w volume on n_sms SMs (the grid is one CTA per SM, or fewer so that a range holds at
    least 64 rows)."""
    n_strips = -(-w // STRIP)
    total = z * n_strips * h
    grid = max(1, min(n_sms, (total + 63) // 64))
    seams = []
    for b in range(1, grid):
        r = total * b // grid
        col, y = divmod(r, h)
        zi, strip = divmod(col, n_strips)
        seams.append((zi, y, strip))
    return seams


def test_fp8_full_size_sampled_and_range_seams():
    """1024x1024x32 in the bench's launch configuration (calibrated on its first 4 slices): 2 seeded
    slices in full vs the oracle; pixels on both sides of every CTA-range seam, at the first and
    last column of the seam's strip, and at slice corners and strip seams, vs the oracle's patch
    form."""
    import torch
    v = synth.em_volume(synth.BASE_SEED + 1, 32, 1024, 1024)
    net = calibrated(v)
    p = infer(net, v)
    params = teacher_params()
    rng = np.random.default_rng(5)
    for zi in rng.choice(32, size=2, replace=False):
        check_fp8(p[zi], oracle.forward_region(T, params, v[zi]), ("slice", zi))
    n_sms = torch.cuda.get_device_properties(0).multi_processor_count
    seams = range_seams(32, 1024, 1024, n_sms)
    assert len(seams) >= min(n_sms, 100) - 1
    pts = set()
    for zi, y, strip in seams:
        x0, x1 = strip * STRIP, min(strip * STRIP + STRIP - 1, 1023)
        for yy in (y - 1, y):
            if 0 <= yy < 1024:
                pts.update({(zi, yy, x0), (zi, yy, x1)})
    for zi in range(0, 32, 7):
        pts.update({(zi, 0, 0), (zi, 0, 1023), (zi, 1023, 0), (zi, 1023, 1023), (zi, 511, 117), (zi, 511, 118)})
    err = [abs(float(p[zi, i, j]) - oracle.patch_pixel(T, params, v[zi], i, j)) for zi, i, j in sorted(pts)]
    assert max(err) <= TOL["fp8"]["max_abs"], max(err)
    assert np.mean(err) <= TOL["fp8"]["mean_abs"], np.mean(err)
    net.close()


def test_fp8_batch_equals_per_block_and_volume(fp8):
    """Uneven blocks in one persistent launch (ranges cross block boundaries) == per-block
    launches == per-volume calls, bitwise; pitch padding untouched."""
    import torch
    from paper_1612_02120_gb300 import membrane as m
    from test_gpu_batch import make_blocks
    shapes = [(2, 37, 300), (1, 256, 129), (3, 64, 64), (1, 8, 8), (2, 120, 250), (1, 300, 40)]
    vols, ins, outs, blocks = make_blocks(shapes, 6201, pitch_pad=5)
    m.mb_infer_batch(fp8.handle, blocks)
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    for o in outs:
        o.fill_(-1.0)
    m.mb_infer_batch(fp8.handle, blocks)  # graph replay
    torch.cuda.synchronize()
    for a, b in zip(first, outs):
        assert torch.equal(a, b)
    _, _, outs_pb, blocks_pb = make_blocks(shapes, 6201, pitch_pad=5)
    m.mb_infer_batch_per_block(fp8.handle, blocks_pb)
    torch.cuda.synchronize()
    for (d, h, w), v, a, b in zip(shapes, vols, outs, outs_pb):
        assert torch.equal(a[:, :, :w], b[:, :, :w])
        assert bool((a[:, :, w:] == -1.0).all())
        np.testing.assert_array_equal(a[:, :, :w].cpu().numpy(), infer(fp8, v))
    check_fp8(outs[1][0, :, :129].cpu().numpy(), oracle.forward_region(T, teacher_params(), vols[1][0]), "block 1")


def test_fp8_host_streaming_equals_device_path():
    """1024x1024x30 from pinned host buffers, in slabs (4, 8, 8, 6, 4 slices on two compute
    streams) and accessed directly by the kernel, equals the device-resident FP8 call bitwise."""
    import torch
    from paper_1612_02120_gb300 import membrane as m
    z = 30
    v = synth.em_volume(6301, z, 1024, 1024)
    net = calibrated(v)
    dev = infer(net, v)
    pin_in = torch.from_numpy(v).pin_memory()
    pin_out = torch.empty((z, 1024, 1024), dtype=torch.float32).pin_memory()
    for mode in (m.MB_HOST_IO_SLABS, m.MB_HOST_IO_SLABS, m.MB_HOST_IO_AUTO):
        m.mb_set_host_io(net.handle, mode)
        pin_out.fill_(-1.0)
        m.mb_infer_volume(net.handle, pin_in, z, 1024, 1024, pin_out)
        np.testing.assert_array_equal(pin_out.numpy(), dev)
    net.close()
