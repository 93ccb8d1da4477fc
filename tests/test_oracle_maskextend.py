"""Pins of the oracle's MaskExtend (Sec. 3.2) to facts outside the oracle: the printed 109x109
field of view, the patch calculation with real stride-2 max-pooling on the 12-map input, the
3-class softmax against numpy, the smoothing-and-thresholding J against scipy, and the
recursion of the transfer equation step by step. CPU only."""
import numpy as np
import pytest

import oracle
import synth
from test_oracle_fastmemb import np_conv, np_maxout, np_maxpool2_stride2
from test_oracle_pins import split_params

M = synth.MASKEXTEND


def me_params():
    return synth.init_params(M, synth.MASKEXTEND_WEIGHT_SEED).astype(np.float64)


def inputs(z=10, h=40, w=36, seed=8100):
    em = synth.em_volume(seed, z, h, w)
    memb = synth.membrane_maps(em)
    seeds = synth.disk_masks(4, h, w, h / 2, w / 2, min(h, w) / 4, 0.5, -0.5)
    return em, memb, seeds


def np_softmax(z):
    e = np.exp(z - z.max(axis=0, keepdims=True))
    return e / e.sum(axis=0)


def test_field_of_view_109_and_parameters():
    """Four conv/pool pairs and a fifth conv of 4x4 kernels: 109x109 (printed: 109)."""
    assert oracle.net_radius(M) == 54
    assert oracle.param_count(M) == synth.param_count(M) == 316067
    n = 109
    for _ in range(4):
        n = (n - 3) // 2
    assert n - 3 == 1


def test_input_stack_channel_order():
    em, memb, seeds = inputs()
    x = oracle.maskextend_input(em, memb, {3 + i: seeds[i] for i in range(4)}, 7, 3)
    assert x.shape == (12, 40 + 6, 36 + 6)
    c = x[:, 3:-3, 3:-3]
    np.testing.assert_array_equal(c[0:3], em[6:9] / 255.0)
    np.testing.assert_array_equal(c[3:7], seeds.astype(np.float64))
    np.testing.assert_array_equal(c[7:12], memb[5:10].astype(np.float64))


def test_dense_equals_patch_calculation_on_the_12_map_stack():
    prm = me_params()
    parts = split_params(M, prm)
    em, memb, seeds = inputs(h=44, w=41)
    xp = oracle.maskextend_input(em, memb, {3 + i: seeds[i] for i in range(4)}, 7, 54)
    dense = oracle.run_layers_mc(M, prm, xp)
    assert dense.shape == (3, 44, 41)
    np.testing.assert_allclose(dense.sum(axis=0), 1.0, rtol=0, atol=1e-12)
    rng = np.random.default_rng(90)
    pix = [(0, 0), (43, 40), (22, 20)] + [tuple(int(v) for v in rng.integers(0, (44, 41))) for _ in range(5)]
    for i, j in pix:
        x = xp[:, i:i + 109, j:j + 109]
        for W, b in parts[:4]:
            x = np_maxpool2_stride2(np_maxout(np_conv(x, W, b), 2))
        x = np_maxout(np_conv(x, *parts[4]), 2)
        assert x.shape == (64, 1, 1)
        W5, b5 = parts[5]
        p = np_softmax(np.einsum("oc,chw->ohw", W5[:, :, 0, 0], x) + b5[:, None, None])
        np.testing.assert_allclose(p[:, 0, 0], dense[:, i, j], rtol=0, atol=1e-12)


def test_smooth_threshold_matches_scipy():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(91)
    p = rng.random((23, 31))
    for thr in (0.3, 0.5, 0.7):
        ref = (ndimage.uniform_filter(p, size=3, mode="mirror") >= thr).astype(np.uint8)
        got = oracle.smooth_threshold(p, thr)
        near = np.abs(ndimage.uniform_filter(p, size=3, mode="mirror") - thr) < 1e-12
        assert np.array_equal(got[~near], ref[~near])


def test_recursion_feeds_each_mask_into_the_next_step():
    prm = me_params()
    em, memb, seeds = inputs(z=10, h=30, w=28)
    masks, probs = oracle.mask_extend(M, prm, em, memb, seeds, 6, 2)
    assert masks.shape == (2, 30, 28) and probs.shape == (2, 3, 30, 28)
    # step 1 by hand: its mask stack holds seeds 3, 4, 5 and the step-0 mask (section 6)
    known = {2 + i: seeds[i] for i in range(4)}
    known[6] = masks[0]
    p7 = oracle.run_layers_mc(M, prm, oracle.maskextend_input(em, memb, known, 7, 54))
    np.testing.assert_array_equal(p7, probs[1])
    np.testing.assert_array_equal(oracle.smooth_threshold(p7[0]), masks[1])
    # a different step-0 mask changes step 1
    known[6] = 1 - masks[0]
    alt = oracle.run_layers_mc(M, prm, oracle.maskextend_input(em, memb, known, 7, 54))
    assert not np.array_equal(alt, probs[1])


def test_input_stack_sections_minus_z():
    """Extending in z- (Sec. 3.2: the algorithm continues in either z+ or z-) mirrors every offset
    of the transfer equation: at section 5 the stack holds EM 6, 5, 4, the masks of the sections
    already extended, 9, 8, 7, 6, and the membrane maps 7, 6, 5, 4, 3, in that channel order."""
    em, memb, seeds = inputs()
    known = {9: seeds[0], 8: seeds[1], 7: seeds[2], 6: seeds[3]}
    x = oracle.maskextend_input(em, memb, known, 5, 2, direction=-1)
    c = x[:, 2:-2, 2:-2]
    np.testing.assert_array_equal(c[0:3], em[[6, 5, 4]] / 255.0)
    np.testing.assert_array_equal(c[3:7], seeds.astype(np.float64))
    np.testing.assert_array_equal(c[7:12], memb[[7, 6, 5, 4, 3]].astype(np.float64))


def test_minus_z_recursion_is_plus_z_on_the_reversed_stack():
    """The z- recursion from z0 equals the z+ recursion on the stack read backwards, from the
    mirrored section, with the same seeds (their order is along the direction of travel)."""
    prm = me_params()
    em, memb, seeds = inputs(z=10, h=30, w=28, seed=8150)
    m_dn, p_dn = oracle.mask_extend(M, prm, em, memb, seeds, 6, 3, direction=-1)
    m_up, p_up = oracle.mask_extend(M, prm, em[::-1].copy(), memb[::-1].copy(), seeds, 10 - 1 - 6, 3)
    np.testing.assert_array_equal(m_dn, m_up)
    np.testing.assert_array_equal(p_dn, p_up)
    # and it is not the z+ recursion from the same section (the direction matters)
    _, p_same = oracle.mask_extend(M, prm, em, memb, seeds, 6, 1)
    assert np.abs(p_same[0] - p_dn[0]).max() > 1e-3
