"""mb_infer_volume_noalloc: the FP32 path for callers that cannot allocate device memory once they
run, because their memory budget is fixed at start-up or because the synchronisation that
cudaMalloc/cudaFree may cause would stall their other streams. Checked through the C ABI against
mb_infer_volume, bitwise (the same three kernels compute every pixel with the same arithmetic),
on two calls in a row and on shapes that run the row-band loop and the slice-chunk loop of its
fixed 64 MiB scratch array. Collected last on purpose."""
import numpy as np
import pytest

import synth
from _common import make_net, teacher_params

pytestmark = pytest.mark.gpu

SCRATCH_FLOATS = (64 << 20) // 4   # the documented 64 MiB scratch


def band_floats(nz, rows, w):
    """Scratch floats of a band of `rows` output rows of nz slices, as the header documents it."""
    return nz * ((rows + 10) * (w + 10) + (rows + 5) * (w + 5)) * 32


def expected_launches(z, h, w):
    """Three launches per band: the largest band of one slice that fits, then as many slices of
    that band as fit per band launch sequence."""
    rows = max(r for r in range(1, h + 1) if band_floats(1, r, w) <= SCRATCH_FLOATS)
    nz = max(1, min(z, SCRATCH_FLOATS // band_floats(1, rows, w)))
    n_chunks = -(-z // nz)
    n_bands = -(-h // rows)
    return 3 * n_chunks * n_bands, rows, nz


def _compare(m, lib, net, z, h, w, seed, out_type, check_launches=True):
    import torch
    v = synth.em_volume(seed, z, h, w)
    x = torch.from_numpy(v).cuda()
    dt = torch.float32 if out_type == m.MB_OUT_F32 else torch.uint8
    ref = torch.empty((z, h, w), dtype=dt, device="cuda")
    got = torch.full((z, h, w), 7, dtype=dt, device="cuda")
    m.mb_infer_volume(net.handle, x, z, h, w, ref, out_type)
    torch.cuda.synchronize()
    l0 = m.launch_count()
    st = lib.mb_infer_volume_noalloc(net.handle, x.data_ptr(), z, h, w, got.data_ptr(), out_type, None)
    assert st == m.MB_OK, m.last_error()
    launched = m.launch_count() - l0
    torch.cuda.synchronize()
    assert torch.equal(got, ref), (z, h, w, out_type, (got.float() - ref.float()).abs().max().item())
    if check_launches:
        want, rows, nz = expected_launches(z, h, w)
        assert launched == want, (launched, want, rows, nz)
    return launched


def test_noalloc_matches_infer_volume_twice():
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    lib = m.load()
    net = make_net(synth.TEACHER, m.MB_PREC_FP32, teacher_params())
    for call, (z, h, w) in enumerate([(3, 200, 170), (2, 96, 130)]):
        _compare(m, lib, net, z, h, w, 5000 + call, m.MB_OUT_F32)
    net.close()


@pytest.mark.parametrize("out_type", [0, 1])
def test_noalloc_row_bands(out_type):
    """A wide slice (about 5 rows per band: 13 bands) and a 2048x2048 volume (about 120 rows per
    band, one slice per chunk): the band edges' layer-1 offsets and the bands' output offsets."""
    from paper_1612_02120_gb300 import membrane as m
    lib = m.load()
    net = make_net(synth.TEACHER, m.MB_PREC_FP32, teacher_params())
    n = _compare(m, lib, net, 2, 64, 20000, 5100, out_type)
    assert n >= 3 * 2 * 10
    n = _compare(m, lib, net, 2, 2048, 2048, 5101, out_type)
    assert n >= 3 * 2 * 16
    net.close()


@pytest.mark.parametrize("out_type", [0, 1])
def test_noalloc_slice_chunks(out_type):
    """Whole slices, three per chunk, and a ragged last chunk (40 = 13 x 3 + 1); then two row bands
    per slice with one slice per chunk (40 x 512 x 512)."""
    from paper_1612_02120_gb300 import membrane as m
    lib = m.load()
    net = make_net(synth.TEACHER, m.MB_PREC_FP32, teacher_params())
    _, rows, nz = expected_launches(40, 256, 256)
    assert rows == 256 and 1 < nz < 40 and 40 % nz != 0
    _compare(m, lib, net, 40, 256, 256, 5200, out_type)
    _, rows, nz = expected_launches(40, 512, 512)
    assert rows < 512 and nz == 1
    _compare(m, lib, net, 40, 512, 512, 5201, out_type)
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
    # taller than 2^20 rows: rejected before any device work (the buffers are never touched)
    assert lib.mb_infer_volume_noalloc(net.handle, x.data_ptr(), 1, (1 << 20) + 1, 16, out.data_ptr(), 0, None) == \
        m.MB_ERR_SHAPE
    assert "2^20" in m.last_error()
    net.close()
