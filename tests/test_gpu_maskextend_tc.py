"""MaskExtend (Sec. 3.2) on the tensor cores (FP16 operands, FP32 accumulation) vs the FP64
oracle, through the C ABI: the 3 class maps of a step within the 16-bit bar, the masks J makes
equal wherever the oracle's smoothed object probability is clear of the threshold by more than
the bar, each step of the +z recursion against the oracle fed the GPU's own earlier masks, the
FP16 path against the FP32 path, the reported device-side wait limit, and the precision rules."""
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
def net16():
    from paper_1612_02120_gb300 import build, membrane as m
    build.build()
    n = make_net(M, m.MB_PREC_FP16, me_params())
    yield n
    n.close()


def data(z, h, w, seed):
    em = synth.em_volume(seed, z, h, w)
    memb = synth.membrane_maps(em)
    seeds = synth.disk_masks(4, h, w, h / 2, w / 2, min(h, w) / 4, 1.0, -0.5)
    return em, memb, seeds


def run_gpu(net, em, memb, seeds, z0, n, probs=True):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    Z, h, w = em.shape
    d_em, d_memb, d_seeds = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (em, memb, seeds))
    masks = torch.zeros((n, h, w), dtype=torch.uint8, device="cuda")
    pr = torch.zeros((n, 3, h, w), dtype=torch.float32, device="cuda") if probs else None
    m.mb_mask_extend(net.handle, d_em, d_memb, Z, h, w, d_seeds, z0, n, masks, pr)
    torch.cuda.synchronize()
    return masks.cpu().numpy(), (pr.cpu().numpy() if probs else None)


def margin(p_obj, thr=0.5):
    pp = np.pad(p_obj, 1, mode="reflect")
    s = sum(pp[a:a + p_obj.shape[0], b:b + p_obj.shape[1]] for a in range(3) for b in range(3))
    return np.abs(s / 9.0 - thr)


def check_step(masks_g, probs_g, ref_p):
    met = oracle.metrics(probs_g, ref_p)
    assert met["max_abs"] <= TOL["fp16"]["max_abs"] and met["mean_abs"] <= TOL["fp16"]["mean_abs"], met
    sure = margin(ref_p[0]) > TOL["fp16"]["max_abs"]
    assert np.array_equal(masks_g[sure], oracle.smooth_threshold(ref_p[0])[sure])


@pytest.mark.parametrize("shape", [(8, 55, 55), (10, 60, 70), (10, 57, 530), (8, 301, 259)])
def test_fp16_recursion_steps_match_oracle(net16, shape):
    """Two steps (one on the widest); the oracle's step s reads the GPU's masks of the earlier
    steps. 55x55 is the smallest section; 530 columns span 5 strips of 128 with a ragged tail."""
    z, h, w = shape
    em, memb, seeds = data(z, h, w, 9200 + h * w)
    z0, n = 4, 1 if w > 300 or h > 300 else 2
    masks, probs = run_gpu(net16, em, memb, seeds, z0, n)
    prm = me_params().astype(np.float64)
    known = {z0 - 4 + i: seeds[i] for i in range(4)}
    for s in range(n):
        ref_p = oracle.run_layers_mc(M, prm, oracle.maskextend_input(em, memb, known, z0 + s, 54))
        check_step(masks[s], probs[s], ref_p)
        known[z0 + s] = masks[s]
    assert masks.max() == 1 and masks.min() == 0


def test_fp16_free_running_recursion_agrees_with_fp32_path(net16):
    """Four free-running steps of the FP16 and FP32 paths on one window. The first step reads the
    same inputs on both: probabilities within the 16-bit bar, masks equal on >= 99.9 % of pixels.
    Later steps read each path's own earlier masks, so a pixel flipped near the threshold changes
    the next four steps' inputs and the paths drift apart: >= 99 % over the four steps."""
    from paper_1612_02120_gb300 import membrane as m
    em, memb, seeds = data(10, 96, 200, 9300)
    m16, p16 = run_gpu(net16, em, memb, seeds, 3, 4)
    with make_net(M, m.MB_PREC_FP32, me_params()) as n32:
        m32, p32 = run_gpu(n32, em, memb, seeds, 3, 4)
    assert np.abs(p16[0] - p32[0]).max() <= TOL["fp16"]["max_abs"]
    assert (m16[0] == m32[0]).mean() >= 0.999
    assert (m16 == m32).mean() >= 0.99


def test_fp16_without_probability_output_gives_the_same_masks(net16):
    em, memb, seeds = data(8, 70, 90, 9400)
    a, _ = run_gpu(net16, em, memb, seeds, 3, 2)
    b, _ = run_gpu(net16, em, memb, seeds, 3, 2, probs=False)
    np.testing.assert_array_equal(a, b)


def test_fp16_repeatable(net16):
    em, memb, seeds = data(8, 66, 140, 9500)
    a = run_gpu(net16, em, memb, seeds, 3, 2)
    b = run_gpu(net16, em, memb, seeds, 3, 2)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_fp16_timed_out_device_wait_is_reported_and_context_survives(net16, monkeypatch):
    import torch
    from paper_1612_02120_gb300 import membrane as m
    lib = m.load()
    em, memb, seeds = data(6, 60, 60, 9600)
    ref_m, _ = run_gpu(net16, em, memb, seeds, 3, 1)
    d_em, d_memb, d_seeds = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (em, memb, seeds))
    out = torch.zeros((1, 60, 60), dtype=torch.uint8, device="cuda")
    call = lambda: lib.mb_mask_extend(net16.handle, d_em.data_ptr(), d_memb.data_ptr(), 6, 60, 60,
                                      d_seeds.data_ptr(), 3, 1, 0.5, out.data_ptr(), None, None)
    monkeypatch.setenv("MB_FAULT_STALL", "1")
    assert call() == m.MB_OK
    torch.cuda.synchronize()
    monkeypatch.delenv("MB_FAULT_STALL")
    assert call() == m.MB_ERR_TIMEOUT
    assert "wait limit" in m.last_error()
    assert call() == m.MB_OK
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref_m)


def test_fp16_is_maskextend_and_fastmemb_only():
    from paper_1612_02120_gb300 import membrane as m
    for layers in (synth.TEACHER, synth.STUDENT):
        with pytest.raises(m.MembraneError) as e:
            m.mb_net_create(layers, m.MB_PREC_FP16, 0)
        assert e.value.status == m.MB_ERR_UNSUPPORTED
    with pytest.raises(m.MembraneError) as e:
        m.mb_net_create(M, m.MB_PREC_BF16, 0)
    assert e.value.status == m.MB_ERR_UNSUPPORTED


def test_fp16_step_at_bench_size_on_sampled_crops(net16):
    """One step on the 512x512 window the bench times, in its launch configuration: the class
    maps of two 96x96 crops (one at a corner, so the mirror padding is inside it) against the
    oracle evaluated on the crops with their true context."""
    em, memb, seeds = data(8, 512, 512, 9700)
    masks, probs = run_gpu(net16, em, memb, seeds, 3, 1)
    prm = me_params().astype(np.float64)
    xp = oracle.maskextend_input(em, memb, {-1 + i: seeds[i] for i in range(4)}, 3, 54)
    for y0, x0 in ((0, 0), (300, 181)):
        ref = oracle.run_layers_mc(M, prm, xp[:, y0:y0 + 96 + 108, x0:x0 + 96 + 108])
        met = oracle.metrics(probs[0][:, y0:y0 + 96, x0:x0 + 96], ref)
        assert met["max_abs"] <= TOL["fp16"]["max_abs"] and met["mean_abs"] <= TOL["fp16"]["mean_abs"], met


def test_fp16_minus_z_steps_match_oracle(net16):
    """The z- recursion on the tensor cores: each step against the oracle's z- step fed the GPU's
    own earlier masks, at the 16-bit bar."""
    import torch
    from paper_1612_02120_gb300 import membrane as m
    em, memb, seeds = data(9, 72, 140, 8800)
    Z, h, w = em.shape
    z0, n = 6, 3
    d_em, d_memb, d_seeds = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (em, memb, seeds))
    masks = torch.zeros((n, h, w), dtype=torch.uint8, device="cuda")
    pr = torch.zeros((n, 3, h, w), dtype=torch.float32, device="cuda")
    m.mb_mask_extend_dir(net16.handle, d_em, d_memb, Z, h, w, d_seeds, z0, n, -1, masks, pr)
    torch.cuda.synchronize()
    masks, pr = masks.cpu().numpy(), pr.cpu().numpy()
    prm = me_params().astype(np.float64)
    known = {z0 + 4 - i: seeds[i] for i in range(4)}
    for s in range(n):
        ref_p = oracle.run_layers_mc(M, prm, oracle.maskextend_input(em, memb, known, z0 - s, 54, direction=-1))
        check_step(masks[s], pr[s], ref_p)
        known[z0 - s] = masks[s]
