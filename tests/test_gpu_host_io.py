"""Host-buffer volumes through mb_infer_volume: direct access (the kernels read the page-locked
input and write the page-locked maps over the coherent CPU-GPU link) and z-slabs through device
buffers must both give the device-resident call's maps bitwise, for every net family. Calls go
through the C ABI."""
import numpy as np
import pytest

import synth
from _common import infer, make_net, student_params, teacher_params

pytestmark = pytest.mark.gpu


def _fm_params():
    return synth.init_params(synth.FASTMEMB, synth.FASTMEMB_WEIGHT_SEED)


def _net(kind):
    import torch
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    if kind == "teacher_bf16":
        return make_net(synth.TEACHER, m.MB_PREC_BF16, teacher_params())
    if kind == "teacher_fp32":
        return make_net(synth.TEACHER, m.MB_PREC_FP32, teacher_params())
    if kind == "teacher_fp8":
        n = make_net(synth.TEACHER, m.MB_PREC_FP8, teacher_params())
        cal = torch.from_numpy(synth.em_volume(synth.BASE_SEED + 3, 4, 256, 256)).cuda()
        m.mb_calibrate_fp8(n.handle, cal, 4, 256, 256)
        return n
    if kind == "student_bf16":
        return make_net(synth.STUDENT, m.MB_PREC_BF16, student_params())
    if kind == "student_fp32":
        return make_net(synth.STUDENT, m.MB_PREC_FP32, student_params())
    if kind == "fastmemb_bf16":
        return make_net(synth.FASTMEMB, m.MB_PREC_BF16, _fm_params())
    raise ValueError(kind)


def _launches(fn):
    from paper_1612_02120_gb300 import membrane as m
    a = m.launch_count()
    fn()
    return m.launch_count() - a


@pytest.mark.parametrize("kind", ["teacher_bf16", "teacher_fp8", "teacher_fp32", "student_bf16",
                                  "student_fp32", "fastmemb_bf16"])
@pytest.mark.parametrize("out_type", [0, 1])
def test_direct_and_slab_host_io_equal_device_path(kind, out_type):
    """4 x 192 x 200 (a ragged strip and row tail for every kernel) from pinned buffers, in both
    host I/O modes; the default mode (direct access; slabs for student nets) makes exactly the
    device path's launches (one slab here)."""
    import torch
    from paper_1612_02120_gb300 import membrane as m
    net = _net(kind)
    z, h, w = 4, 192, 200
    v = synth.em_volume(7100, z, h, w)
    dev = infer(net, v, out_type)
    dev_launches = _launches(lambda: infer(net, v, out_type))
    pin_in = torch.from_numpy(v).pin_memory()
    pin_out = torch.empty((z, h, w), dtype=torch.float32 if out_type == 0 else torch.uint8).pin_memory()
    for mode in (m.MB_HOST_IO_AUTO, m.MB_HOST_IO_SLABS, m.MB_HOST_IO_AUTO):
        m.mb_set_host_io(net.handle, mode)
        pin_out.fill_(7)
        n = _launches(lambda: m.mb_infer_volume(net.handle, pin_in, z, h, w, pin_out, out_type))
        np.testing.assert_array_equal(pin_out.numpy(), dev)
        if mode == m.MB_HOST_IO_AUTO:
            assert n == dev_launches
    net.close()


def test_direct_host_io_at_interior_offsets_and_mixed_buffers():
    """Views that start inside a pinned allocation (slice offsets) are accessed at their own
    address; a pinned input with a pageable output (not mapped) streams in slabs; both equal the
    device path bitwise, and the slab path launches once per slab."""
    import torch
    from paper_1612_02120_gb300 import membrane as m
    net = _net("teacher_bf16")
    z, h, w = 12, 1024, 1024  # above one 8-slice slab, so the slab path launches twice
    v = synth.em_volume(7200, z + 3, h, w)
    dev = infer(net, v[3:])
    big_in = torch.from_numpy(v).pin_memory()
    big_out = torch.full((z + 2, h, w), -1.0, dtype=torch.float32).pin_memory()
    view_in, view_out = big_in[3:], big_out[2:]
    assert view_in.is_contiguous() and view_out.is_contiguous()
    n = _launches(lambda: m.mb_infer_volume(net.handle, view_in, z, h, w, view_out))
    assert n == 1
    np.testing.assert_array_equal(view_out.numpy(), dev)
    assert (big_out[:2] == -1.0).all()  # nothing written before the view
    pageable_out = np.full((z, h, w), -1.0, dtype=np.float32)
    n = _launches(lambda: m.mb_infer_volume(net.handle, view_in, z, h, w, pageable_out))
    assert n > 1
    np.testing.assert_array_equal(pageable_out, dev)
    net.close()


def test_host_io_mode_is_validated():
    from paper_1612_02120_gb300 import membrane as m
    net = _net("student_bf16")
    lib = m.load()
    assert lib.mb_set_host_io(net.handle, 2) == m.MB_ERR_INVALID_ARG
    assert lib.mb_set_host_io(net.handle, -1) == m.MB_ERR_INVALID_ARG
    assert lib.mb_set_host_io(None, 0) == m.MB_ERR_INVALID_ARG
    assert lib.mb_set_host_io(net.handle, m.MB_HOST_IO_SLABS) == m.MB_OK
    net.close()
