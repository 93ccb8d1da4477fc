"""MaskExtend (Sec. 3.2) on the FP32 CUDA-core path vs the FP64 oracle, through the C ABI: the
3 class maps of a step within 1e-5 max-abs; the masks J makes equal wherever the oracle's smoothed
object probability is more than 1e-4 from the threshold (FP32 cannot decide closer ones the same
way); each step of the +z recursion checked against the oracle fed the GPU's own earlier masks;
a free-running recursion; and the error codes."""
import numpy as np
import pytest

import oracle
import synth
from _common import TOL, make_net

pytestmark = pytest.mark.gpu

M = synth.MASKEXTEND


def me_params():
    return synth.init_params(M, synth.MASKEXTEND_WEIGHT_SEED)


@pytest.fixture(scope="module")
def net():
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    n = make_net(M, m.MB_PREC_FP32, me_params())
    yield n
    n.close()


def data(z, h, w, seed):
    em = synth.em_volume(seed, z, h, w)
    memb = synth.membrane_maps(em)
    seeds = synth.disk_masks(4, h, w, h / 2, w / 2, min(h, w) / 4, 1.0, -0.5)
    return em, memb, seeds


def run_gpu(net, em, memb, seeds, z0, n):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    Z, h, w = em.shape
    d_em, d_memb, d_seeds = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (em, memb, seeds))
    masks = torch.zeros((n, h, w), dtype=torch.uint8, device="cuda")
    probs = torch.zeros((n, 3, h, w), dtype=torch.float32, device="cuda")
    m.mb_mask_extend(net.handle, d_em, d_memb, Z, h, w, d_seeds, z0, n, masks, probs)
    torch.cuda.synchronize()
    return masks.cpu().numpy(), probs.cpu().numpy()


def margin(p_obj, thr=0.5):
    """|3x3 mean (reflect-101) - thr| of the oracle's object map."""
    pp = np.pad(p_obj, 1, mode="reflect")
    s = sum(pp[a:a + p_obj.shape[0], b:b + p_obj.shape[1]] for a in range(3) for b in range(3))
    return np.abs(s / 9.0 - thr)


def check_step(masks_g, probs_g, ref_p):
    assert oracle.metrics(probs_g, ref_p)["max_abs"] <= TOL["fp32"]["max_abs"]
    ref_m = oracle.smooth_threshold(ref_p[0])
    sure = margin(ref_p[0]) > 1e-4
    assert np.array_equal(masks_g[sure], ref_m[sure])
    return int((~sure).sum())


@pytest.mark.parametrize("shape", [(10, 60, 70), (10, 57, 530)])
def test_recursion_steps_match_oracle(net, shape):
    """Three steps; the oracle's step s reads the GPU's masks of the earlier steps."""
    z, h, w = shape
    em, memb, seeds = data(z, h, w, 8200 + h * w)
    z0, n = 4, 2 if w > 300 else 3
    masks, probs = run_gpu(net, em, memb, seeds, z0, n)
    prm = me_params().astype(np.float64)
    known = {z0 - 4 + i: seeds[i] for i in range(4)}
    for s in range(n):
        ref_p = oracle.run_layers_mc(M, prm, oracle.maskextend_input(em, memb, known, z0 + s, 54))
        check_step(masks[s], probs[s], ref_p)
        known[z0 + s] = masks[s]
    assert masks.max() == 1 and masks.min() == 0


def test_free_running_recursion_agrees_with_oracle(net):
    em, memb, seeds = data(9, 64, 72, 8300)
    masks, probs = run_gpu(net, em, memb, seeds, 3, 4)
    ref_m, ref_p = oracle.mask_extend(M, me_params(), em, memb, seeds, 3, 4)
    assert (masks == ref_m).mean() >= 0.999
    assert oracle.metrics(probs[0], ref_p[0])["max_abs"] <= TOL["fp32"]["max_abs"]


def test_maskextend_error_codes(net):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    lib = m.load()
    em, memb, seeds = data(6, 60, 60, 8400)
    d_em, d_memb, d_seeds = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (em, memb, seeds))
    out = torch.zeros((4, 60, 60), dtype=torch.uint8, device="cuda")
    call = lambda z0, n: lib.mb_mask_extend(net.handle, d_em.data_ptr(), d_memb.data_ptr(), 6, 60, 60,
                                            d_seeds.data_ptr(), z0, n, 0.5, out.data_ptr(), None, None)
    assert call(1, 1) == m.MB_ERR_SHAPE          # needs membrane maps from z0 - 2
    assert call(3, 2) == m.MB_ERR_SHAPE          # the last step needs sections up to z0 + n + 1
    assert call(3, 1) == m.MB_OK
    assert call(3, 0) == m.MB_OK
    torch.cuda.synchronize()
    x = torch.zeros((1, 60, 60), dtype=torch.uint8, device="cuda")
    y = torch.zeros((1, 60, 60), dtype=torch.float32, device="cuda")
    assert lib.mb_infer_volume(net.handle, x.data_ptr(), 1, 60, 60, y.data_ptr(), 0, None) == m.MB_ERR_UNSUPPORTED
    with pytest.raises(m.MembraneError) as e:
        m.mb_net_create(M, m.MB_PREC_BF16, 0)
    assert e.value.status == m.MB_ERR_UNSUPPORTED
    assert net.n_params == 316067


def run_gpu_dir(net, em, memb, seeds, z0, n, direction):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    Z, h, w = em.shape
    d_em, d_memb, d_seeds = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (em, memb, seeds))
    masks = torch.zeros((n, h, w), dtype=torch.uint8, device="cuda")
    probs = torch.zeros((n, 3, h, w), dtype=torch.float32, device="cuda")
    m.mb_mask_extend_dir(net.handle, d_em, d_memb, Z, h, w, d_seeds, z0, n, direction, masks, probs)
    torch.cuda.synchronize()
    return masks.cpu().numpy(), probs.cpu().numpy()


@pytest.mark.parametrize("shape", [(10, 60, 70), (9, 57, 300)])
def test_minus_z_steps_match_oracle(net, shape):
    """The z- recursion (every offset of the transfer equation mirrored): each step against the
    oracle's z- step fed the GPU's own earlier masks."""
    z, h, w = shape
    em, memb, seeds = data(z, h, w, 8500 + h * w)
    z0, n = z - 3, 3
    masks, probs = run_gpu_dir(net, em, memb, seeds, z0, n, -1)
    prm = me_params().astype(np.float64)
    known = {z0 + 4 - i: seeds[i] for i in range(4)}
    for s in range(n):
        ref_p = oracle.run_layers_mc(M, prm, oracle.maskextend_input(em, memb, known, z0 - s, 54, direction=-1))
        check_step(masks[s], probs[s], ref_p)
        known[z0 - s] = masks[s]


def test_minus_z_is_plus_z_on_the_reversed_stack(net):
    """Same kernels on the same maps: z- from z0 equals z+ on the stack read backwards, bitwise."""
    em, memb, seeds = data(9, 64, 72, 8600)
    m_dn, p_dn = run_gpu_dir(net, em, memb, seeds, 6, 4, -1)
    m_up, p_up = run_gpu_dir(net, em[::-1].copy(), memb[::-1].copy(), seeds, 9 - 1 - 6, 4, 1)
    np.testing.assert_array_equal(m_dn, m_up)
    np.testing.assert_array_equal(p_dn, p_up)
    m_plain, p_plain = run_gpu(net, em[::-1].copy(), memb[::-1].copy(), seeds, 2, 4)
    np.testing.assert_array_equal(p_plain, p_up)   # mb_mask_extend is direction +1


def test_minus_z_error_codes(net):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    lib = m.load()
    em, memb, seeds = data(6, 60, 60, 8700)
    d_em, d_memb, d_seeds = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (em, memb, seeds))
    out = torch.zeros((4, 60, 60), dtype=torch.uint8, device="cuda")
    call = lambda z0, n, d: lib.mb_mask_extend_dir(net.handle, d_em.data_ptr(), d_memb.data_ptr(), 6, 60, 60,
                                                   d_seeds.data_ptr(), z0, n, d, 0.5, out.data_ptr(), None, None)
    assert call(4, 1, -1) == m.MB_ERR_SHAPE       # needs membrane maps up to z0 + 2
    assert call(2, 2, -1) == m.MB_ERR_SHAPE       # the last step needs sections down to z0 - n - 1
    assert call(3, 0, 2) == m.MB_ERR_INVALID_ARG  # direction must be +1 or -1
    assert call(3, 2, -1) == m.MB_OK
    assert call(2, 1, -1) == m.MB_OK
    torch.cuda.synchronize()
