"""FastMemb in dense form (Sec. 2.2) on the FP32 CUDA-core path vs the FP64 oracle, element by
element (max-abs <= 1e-5), at sizes that span several fragment tiles at every dilation with
ragged tails; sampled pixels of a full 1024x1024 slice against the oracle's patch calculation;
and the path's invariants and error codes. Calls go through the C ABI."""
import numpy as np
import pytest

import oracle
import synth
from _common import TOL, infer, make_net, within

pytestmark = pytest.mark.gpu

F = synth.FASTMEMB


def fm_params():
    return synth.init_params(F, synth.FASTMEMB_WEIGHT_SEED)


@pytest.fixture(scope="module")
def net():
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    n = make_net(F, m.MB_PREC_FP32, fm_params())
    yield n
    n.close()


def test_param_count_through_the_abi(net):
    assert net.n_params == 67778 == oracle.param_count(F)


@pytest.mark.parametrize("shape", [(1, 27, 27), (2, 64, 45), (1, 300, 280), (1, 33, 270), (3, 41, 58)])
def test_slices_match_oracle(net, shape):
    z, h, w = shape
    v = synth.em_volume(9000 + h * w, z, h, w)
    p = infer(net, v)
    prm = fm_params()
    for zi in range(z):
        ref = oracle.forward_region(F, prm, v[zi])
        met = oracle.metrics(p[zi], ref)
        assert within(met, TOL["fp32"]), (shape, zi, met)


def test_full_size_slice_sampled_against_patch_calculation(net):
    """A 1024x1024 slice: 40 sampled pixels (corners, edges, random) against the oracle's
    evaluation of each pixel's own 53x53 field of view."""
    s = synth.em_slice(synth.slice_seed(synth.BASE_SEED + 5, 0, 0), 1024, 1024)
    p = infer(net, s[None])[0]
    prm = fm_params()
    rng = np.random.default_rng(11)
    pix = [(0, 0), (0, 1023), (1023, 0), (1023, 1023), (511, 0), (0, 700), (25, 26), (1000, 998)]
    pix += [tuple(int(t) for t in rng.integers(0, 1024, 2)) for _ in range(32)]
    err = max(abs(float(p[i, j]) - oracle.patch_pixel(F, prm, s, i, j)) for i, j in pix)
    assert err <= TOL["fp32"]["max_abs"], err
    assert np.all((p >= 0) & (p <= 1))


def test_region_matches_oracle_region_with_true_context(net):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    v = synth.em_volume(9100, 2, 140, 150)
    x = torch.from_numpy(v).cuda()
    out = torch.empty((2, 50, 61), dtype=torch.float32, device="cuda")
    m.mb_infer_region(net.handle, x, 2, 140, 150, 17, 40, 50, 61, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for zi in range(2):
        ref = oracle.forward_region(F, fm_params(), v[zi], 17, 40, 50, 61)
        assert oracle.metrics(got[zi], ref)["max_abs"] <= TOL["fp32"]["max_abs"]
    np.testing.assert_array_equal(got, infer(net, v)[:, 17:67, 40:101])


def test_u8_output_is_rounded_float_output(net):
    v = synth.em_volume(9200, 2, 64, 96)
    pf = infer(net, v, 0)
    pq = infer(net, v, 1)
    q = np.minimum(255, np.floor(np.float32(255.0) * pf + np.float32(0.5))).astype(np.uint8)
    np.testing.assert_array_equal(pq, q)


def test_host_buffers_and_batch_match_device_path(net):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    v = synth.em_volume(9300, 3, 80, 72)
    dev = infer(net, v)
    host_out = np.empty((3, 80, 72), dtype=np.float32)
    m.mb_infer_volume(net.handle, np.ascontiguousarray(v), 3, 80, 72, host_out)
    np.testing.assert_array_equal(host_out, dev)
    # two blocks with padded pitches through the batch call
    shapes = [(2, 40, 33), (1, 29, 90)]
    blocks, outs, vols = [], [], []
    for i, (d, h, w) in enumerate(shapes):
        vol = synth.em_volume(9301, d, h, w, block=i)
        xi = torch.zeros((d, h, w + 3), dtype=torch.uint8, device="cuda")
        xi[:, :, :w] = torch.from_numpy(vol).cuda()
        o = torch.full((d, h, w + 5), -1.0, dtype=torch.float32, device="cuda")
        blocks.append((xi, d, h, w, w + 3, h * (w + 3), o, w + 5, h * (w + 5)))
        outs.append(o)
        vols.append(vol)
    m.mb_infer_batch(net.handle, blocks)
    torch.cuda.synchronize()
    for (d, h, w), vol, o in zip(shapes, vols, outs):
        o = o.cpu().numpy()
        np.testing.assert_array_equal(o[:, :, :w], infer(net, vol))
        assert (o[:, :, w:] == -1.0).all()


def test_slices_are_independent(net):
    v = synth.em_volume(9400, 3, 48, 40)
    all_ = infer(net, v)
    for zi in range(3):
        np.testing.assert_array_equal(all_[zi], infer(net, v[zi:zi + 1])[0])


def test_error_codes():
    import torch
    from paper_1612_02120_gb300 import membrane as m
    lib = m.load()
    with pytest.raises(m.MembraneError) as e:
        m.mb_net_create(F, m.MB_PREC_BF16, 0)
    assert e.value.status == m.MB_ERR_UNSUPPORTED
    bad = list(F)
    bad[2] = (synth.CONV, 4, 32, 32, 0, 3, 2)  # dilation 3: no kernel
    with pytest.raises(m.MembraneError) as e:
        m.mb_net_create(bad, m.MB_PREC_FP32, 0)
    assert e.value.status == m.MB_ERR_UNSUPPORTED
    n = make_net(F, m.MB_PREC_FP32, fm_params())
    x = torch.zeros((1, 26, 64), dtype=torch.uint8, device="cuda")
    out = torch.empty((1, 26, 64), dtype=torch.float32, device="cuda")
    assert lib.mb_infer_volume(n.handle, x.data_ptr(), 1, 26, 64, out.data_ptr(), 0, None) == m.MB_ERR_SHAPE
    assert lib.mb_infer_volume(n.handle, x.data_ptr(), 1, 64, 26, out.data_ptr(), 0, None) == m.MB_ERR_SHAPE
    n.close()
