"""Pins of the FP64 oracle to facts outside itself: library routines (scipy correlation, numpy
sliding maxima), closed forms, the dense-equals-patch identity of Sec. 2.2 ("Accelerating dense
computation"), impulse responses, locality/equivariance and finite differences.
CPU only."""
import numpy as np
import pytest

import oracle
import synth

T = synth.TEACHER
S = synth.STUDENT


def teacher_params(seed=synth.TEACHER_WEIGHT_SEED):
    return synth.init_params(T, seed).astype(np.float64)


def split_params(layers, params):
    """Unpack a flat parameter vector into [(W, b)] per parameterised layer."""
    out, o = [], 0
    for layer in layers:
        kind, k, cin, cout = layer[:4]
        if kind in (synth.CONV, synth.HEAD_SIGMOID, synth.HEAD_SOFTMAX2, synth.HEAD_SOFTMAX):
            cout *= layer[6] if len(layer) > 6 else 1
            n = cout * cin * k * k
            out.append((params[o:o + n].reshape(cout, cin, k, k), params[o + n:o + n + cout]))
            o += n + cout
    assert o == params.size
    return out


def test_reflect101_index_map():
    n = 10
    assert [oracle.reflect101(t, n) for t in range(-3, 0)] == [3, 2, 1]
    assert [oracle.reflect101(t, n) for t in range(n, n + 3)] == [8, 7, 6]
    assert [oracle.reflect101(t, n) for t in range(n)] == list(range(n))
    # matches numpy's 'reflect' padding mode (reflect-101, edge not repeated)
    row = np.arange(n)
    padded = np.pad(row, 7, mode="reflect")
    assert list(padded) == [oracle.reflect101(t, n) for t in range(-7, n + 7)]


def test_param_count_and_radius():
    assert oracle.param_count(T) == synth.param_count(T) == 52129
    assert oracle.net_radius(T) == 7          # 15x15 receptive field
    assert oracle.net_radius(S) == 2
    assert oracle.param_count(S) == 16 * 9 + 16 + 16 * 16 * 9 + 16 + 16 + 1


def test_conv_matches_scipy_correlate():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 11, 13))
    W = rng.standard_normal((4, 3, 5, 5))
    b = rng.standard_normal(4)
    y = oracle.conv(x, W, b, relu=False)
    ref = np.stack([b[co] + sum(signal.correlate2d(x[ci], W[co, ci], mode="valid") for ci in range(3))
                    for co in range(4)])
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12)
    yr = oracle.conv(x, W, b, relu=True)
    np.testing.assert_allclose(yr, np.maximum(ref, 0.0), rtol=0, atol=1e-12)
    assert (yr == 0).any() and (yr > 0).any()


def test_maxfilter_matches_sliding_window_max():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 7, 9))
    y = oracle.maxfilter2(x)
    ref = np.lib.stride_tricks.sliding_window_view(x, (2, 2), axis=(1, 2)).max(axis=(-1, -2))
    np.testing.assert_array_equal(y, ref)


def test_head_matches_numpy():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((5, 4, 6))
    wv = rng.standard_normal(5)
    p = oracle.head_sigmoid(x, wv, 0.3)
    ref = 1.0 / (1.0 + np.exp(-(0.3 + np.einsum("c,chw->hw", wv, x))))
    np.testing.assert_allclose(p, ref, rtol=0, atol=1e-15)


def test_impulse_reproduces_flipped_kernel():
    """conv5x5 1->1 (no ReLU) + identity head on a single impulse: logit(p) = b + the kernel
    flipped about its centre around the impulse, b elsewhere (cross-correlation)."""
    layers = ((synth.CONV, 5, 1, 1, 0), (synth.HEAD_SIGMOID, 1, 1, 1, 0))
    rng = np.random.default_rng(4)
    Wk = rng.standard_normal((5, 5)) * 0.3
    b = 0.05
    params = np.concatenate([Wk.ravel(), [b], [1.0], [0.0]])
    img = np.zeros((16, 16), dtype=np.uint8)
    img[8, 7] = 255
    p = oracle.forward_region(layers, params, img)
    logit = np.log(p / (1.0 - p))
    expect = np.full((16, 16), b)
    expect[6:11, 5:10] += Wk[::-1, ::-1]
    np.testing.assert_allclose(logit, expect, rtol=0, atol=1e-12)


def closed_form_constant(params, x_const):
    """Constant input image: every layer's map is constant (padding keeps it so)."""
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = split_params(T, params)
    h1 = np.maximum(b1 + x_const * W1.sum(axis=(1, 2, 3)), 0.0)
    h2 = np.maximum(b2 + np.einsum("oikl,i->o", W2, h1), 0.0)
    h3 = np.maximum(b3 + np.einsum("oikl,i->o", W3, h2), 0.0)
    z = b4[0] + W4.reshape(-1) @ h3
    return 1.0 / (1.0 + np.exp(-z))


@pytest.mark.parametrize("value", [0, 255])
def test_constant_input_closed_form(value):
    params = teacher_params()
    img = np.full((12, 10), value, dtype=np.uint8)
    p = oracle.forward_region(T, params, img)
    np.testing.assert_allclose(p, closed_form_constant(params, value / 255.0), rtol=0, atol=1e-13)


@pytest.mark.parametrize("shape", [(8, 8), (9, 11)])
def test_dense_equals_patch_calculation(shape):
    """Sec. 2.2: dense computation yields the labels of the per-pixel patch calculation."""
    params = teacher_params()
    img = synth.em_slice(11, 64, 64)[20:20 + shape[0], 30:30 + shape[1]].copy()
    dense = oracle.forward_region(T, params, img)
    for i in range(shape[0]):
        for j in range(shape[1]):
            assert abs(dense[i, j] - oracle.patch_pixel(T, params, img, i, j)) <= 1e-12


def test_translation_equivariance_and_border_effect():
    params = teacher_params()
    big = synth.em_slice(12, 60, 60)
    a = oracle.forward_region(T, params, big[0:40, 0:40].copy())
    dy, dx = 9, 5
    b = oracle.forward_region(T, params, big[dy:dy + 40, dx:dx + 40].copy())
    # pixels at least 7 px from both crops' borders see identical context
    ia = a[dy + 7:40 - 7, dx + 7:40 - 7]
    ib = b[7:40 - 7 - dy, 7:40 - 7 - dx]
    np.testing.assert_array_equal(ia, ib)
    # within the band the mirror padding matters
    assert np.abs(a[dy:dy + 7, dx:40 - dx] - b[0:7, 0:40 - 2 * dx]).max() > 1e-6


def test_region_equals_full_slice_crop():
    params = teacher_params()
    img = synth.em_slice(13, 48, 52)
    full = oracle.forward_region(T, params, img)
    part = oracle.forward_region(T, params, img, 5, 9, 20, 17)
    np.testing.assert_array_equal(part, full[5:25, 9:26])


def test_receptive_field_is_15x15():
    params = teacher_params()
    img = synth.em_slice(14, 40, 40)
    base = oracle.forward_region(T, params, img)
    bumped = img.copy()
    bumped[20, 20] = 255 - bumped[20, 20]
    p = oracle.forward_region(T, params, bumped)
    changed = np.abs(p - base) > 0
    ys, xs = np.nonzero(changed)
    assert ys.min() >= 13 and ys.max() <= 27 and xs.min() >= 13 and xs.max() <= 27
    assert changed[13, 20] or changed[27, 20] or changed[20, 13] or changed[20, 27]


def test_relu_and_maxfilter_commute():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2, 9, 9))
    W = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    a = oracle.maxfilter2(oracle.conv(x, W, b, relu=True))
    c = np.maximum(oracle.maxfilter2(oracle.conv(x, W, b, relu=False)), 0.0)
    np.testing.assert_array_equal(a, c)


def test_output_is_a_probability_map():
    params = teacher_params()
    img = synth.em_slice(15, 32, 32)
    p = oracle.forward_region(T, params, img)
    assert np.all(p > 0.0) and np.all(p < 1.0)


def test_student_gradient_matches_central_differences():
    rng = np.random.default_rng(6)
    params = synth.init_params(S, synth.STUDENT_WEIGHT_SEED, bias_std=0.05).astype(np.float64)
    imgs = rng.integers(0, 256, size=(2, 6, 6), dtype=np.uint8)
    tgt = rng.uniform(0.1, 0.9, size=(2, 6, 6))
    loss, g = oracle.student_loss_grad(S, params, imgs, tgt)
    h = 1e-6
    idx = list(range(0, params.size, 7)) + [params.size - 1, params.size - 2, 160, 161]
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.student_loss_grad(S, pp, imgs, tgt)[0] - oracle.student_loss_grad(S, pm, imgs, tgt)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), abs(g[i])) + 1e-11, (i, fd, g[i])


def test_centred_layer1_is_the_same_network_on_a_centred_input():
    """c1 = b1 + sum(W1)/2 makes the first layer on the mirror-padded x - 1/2 equal the first
    layer on x with b1 (numpy padding and scipy correlation, not the oracle's loops)."""
    from scipy.signal import correlate2d
    params = synth.init_params(S, synth.STUDENT_WEIGHT_SEED, bias_std=0.05).astype(np.float64)
    th = oracle.centred_layer1(S, params)
    np.testing.assert_array_equal(th[160:], params[160:])
    np.testing.assert_allclose(oracle.plain_layer1(S, th), params, rtol=0, atol=1e-15)
    x = synth.em_slice(21, 11, 13).astype(np.float64) / 255.0
    xp = np.pad(x, 1, mode="reflect")
    xc = np.pad(x - 0.5, 1, mode="reflect")
    W1 = params[:144].reshape(16, 3, 3)
    for co in range(16):
        a = correlate2d(xp, W1[co], mode="valid") + params[144 + co]
        b = correlate2d(xc, W1[co], mode="valid") + th[144 + co]
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


def test_centred_gradient_matches_central_differences():
    """The training update's gradient (layer 1 in centred coordinates) equals central differences
    of the loss as a function of those coordinates."""
    rng = np.random.default_rng(8)
    params = synth.init_params(S, synth.STUDENT_WEIGHT_SEED, bias_std=0.05).astype(np.float64)
    imgs = rng.integers(0, 256, size=(2, 6, 6), dtype=np.uint8)
    tgt = rng.uniform(0.1, 0.9, size=(2, 6, 6))
    _, g = oracle.student_loss_grad(S, params, imgs, tgt)
    gc = oracle.centred_grad(S, g)
    th = oracle.centred_layer1(S, params)

    def loss_c(t):
        return oracle.student_loss_grad(S, oracle.plain_layer1(S, t), imgs, tgt)[0]

    h = 1e-6
    for i in list(range(0, 160)) + [160, 1000, params.size - 1]:
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (loss_c(tp) - loss_c(tm)) / (2 * h)
        assert abs(fd - gc[i]) <= 1e-6 * max(abs(fd), abs(gc[i])) + 1e-11, (i, fd, gc[i])


def test_student_first_update_closed_form():
    """From zero moments every centred coordinate moves by -lr g/(|g| + eps); mapped back, each
    layer-1 bias moves by its own step plus half the sum of its channel's weight steps."""
    rng = np.random.default_rng(9)
    params = synth.init_params(S, synth.STUDENT_WEIGHT_SEED, bias_std=0.05).astype(np.float64)
    g = rng.normal(size=params.size)
    z = np.zeros(params.size)
    w, m, v = oracle.student_adam_step(S, params, z, z, g, step=1, lr=1e-3)
    gw = g[:144].reshape(16, 9) - 0.5 * g[144:160, None]
    dw = 1e-3 * gw / (np.abs(gw) + 1e-8)
    db = 1e-3 * g[144:160] / (np.abs(g[144:160]) + 1e-8)
    np.testing.assert_allclose(w[:144], params[:144] - dw.reshape(-1), rtol=0, atol=1e-14)
    np.testing.assert_allclose(w[144:160], params[144:160] - db + 0.5 * dw.sum(axis=1), rtol=0, atol=1e-14)
    rest = 1e-3 * g[160:] / (np.abs(g[160:]) + 1e-8)
    np.testing.assert_allclose(w[160:], params[160:] - rest, rtol=0, atol=1e-14)
    np.testing.assert_allclose(m[:144], 0.1 * gw.reshape(-1), rtol=1e-14)


def test_student_loss_is_mse():
    params = synth.init_params(S, synth.STUDENT_WEIGHT_SEED).astype(np.float64)
    imgs = synth.em_volume(3, 2, 10, 12)
    tgt = np.random.default_rng(7).uniform(0, 1, size=(2, 10, 12))
    loss, _ = oracle.student_loss_grad(S, params, imgs, tgt)
    p = np.stack([oracle.forward_region(S, params, s) for s in imgs])
    assert abs(loss - np.mean((p - tgt) ** 2)) <= 1e-15


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-9, -3e-7, 0.0])
    w0 = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    z = np.zeros_like(g)
    w, m, v = oracle.adam_step(w0, z, z, g, step=1, lr=1e-3)
    expect = w0 - 1e-3 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(w, expect, rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-15)


def test_adam_constant_gradient_bias_correction():
    """With a constant gradient, bias correction makes mhat = g and vhat = g^2 at every step."""
    g = np.array([0.25, -1.5])
    w = np.zeros(2)
    m = np.zeros(2)
    v = np.zeros(2)
    for t in range(1, 6):
        w, m, v = oracle.adam_step(w, m, v, g, step=t, lr=1e-2)
    expect = -5 * 1e-2 * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(w, expect, rtol=1e-12)


def _centred_student_loss(theta, imgs, tgt):
    """The student written for the centred input x - 1/2 in plain numpy/scipy (no oracle code):
    mirror pad 2 (reflect-101), conv3x3 1->16 + c1, ReLU, conv3x3 16->16 + b2, ReLU, 1x1 + bh,
    sigmoid, mean squared error. theta uses the parameter layout with c1 in place of b1."""
    from scipy.signal import correlate2d
    W1 = theta[:144].reshape(16, 3, 3)
    c1 = theta[144:160]
    W2 = theta[160:2464].reshape(16, 16, 3, 3)
    b2 = theta[2464:2480]
    wh, bh = theta[2480:2496], theta[2496]
    se, n = 0.0, 0
    for img, t in zip(imgs, tgt):
        x = np.pad(img.astype(np.float64) / 255.0 - 0.5, 2, mode="reflect")
        h1 = np.stack([np.maximum(correlate2d(x, W1[c], mode="valid") + c1[c], 0.0) for c in range(16)])
        h2 = np.stack([np.maximum(sum(correlate2d(h1[i], W2[c, i], mode="valid") for i in range(16)) + b2[c], 0.0)
                       for c in range(16)])
        p = 1.0 / (1.0 + np.exp(-(np.tensordot(wh, h2, axes=1) + bh)))
        se += float(((p - t) ** 2).sum())
        n += p.size
    return se / n


def test_centred_update_is_adam_on_the_centred_input_network():
    """Two training updates of the stored network (oracle.student_adam_step) equal two plain Adam
    steps on the network that takes x - 1/2 as input (gradients by central differences, numpy
    only), mapped back by b1 = c1 - sum(W1)/2."""
    rng = np.random.default_rng(11)
    w = synth.init_params(S, synth.STUDENT_WEIGHT_SEED, bias_std=0.05, centred_input=True).astype(np.float64)
    imgs = rng.integers(0, 256, size=(2, 5, 6), dtype=np.uint8)
    tgt = rng.uniform(0.1, 0.9, size=(2, 5, 6))
    th = oracle.centred_layer1(S, w)
    assert abs(_centred_student_loss(th, imgs, tgt) - oracle.student_loss_grad(S, w, imgs, tgt)[0]) <= 1e-13
    m = np.zeros(w.size)
    v = np.zeros(w.size)
    mc = np.zeros(w.size)
    vc = np.zeros(w.size)
    h = 1e-6
    for step in (1, 2):  # from step 2 the moments enter
        _, g = oracle.student_loss_grad(S, w, imgs, tgt)
        w, m, v = oracle.student_adam_step(S, w, m, v, g, step=step, lr=1e-3)
        gc = np.empty(th.size)
        for i in range(th.size):
            tp, tm = th.copy(), th.copy()
            tp[i] += h
            tm[i] -= h
            gc[i] = (_centred_student_loss(tp, imgs, tgt) - _centred_student_loss(tm, imgs, tgt)) / (2 * h)
        mc = 0.9 * mc + 0.1 * gc
        vc = 0.999 * vc + 0.001 * gc * gc
        th = th - 1e-3 * (mc / (1 - 0.9 ** step)) / (np.sqrt(vc / (1 - 0.999 ** step)) + 1e-8)
    # differences of the order of the finite-difference error only (a wrong factor or sign in the
    # change of coordinates moves parameters by ~lr = 1e-3)
    assert np.abs(oracle.plain_layer1(S, th) - w).max() <= 2e-6


def _numpy_teacher_maxfilter_maps(params, slice_u8, y0, x0, h, w):
    """The stand-in teacher up to its second max-filter, written with numpy and scipy only: the
    region's 7-px context (numpy 'reflect' = reflect-101 at the slice borders), scipy correlation
    per channel pair, ReLU, and numpy sliding 2x2 maxima."""
    signal = pytest.importorskip("scipy.signal")
    (W1, b1), (W2, b2) = split_params(T, params)[:2]
    xp = np.pad(slice_u8.astype(np.float64) / 255.0, 7, mode="reflect")[y0:y0 + h + 14, x0:x0 + w + 14]

    def conv_relu(x, W, b):
        return np.maximum(np.stack([b[co] + sum(signal.correlate2d(x[ci], W[co, ci], mode="valid")
                                                for ci in range(W.shape[1])) for co in range(W.shape[0])]), 0.0)

    def maxf(x):
        return np.lib.stride_tricks.sliding_window_view(x, (2, 2), axis=(1, 2)).max(axis=(-1, -2))

    m1 = maxf(conv_relu(xp[None], W1, b1))
    m2 = maxf(conv_relu(m1, W2, b2))
    return m1, m2


@pytest.mark.parametrize("region", [None, (5, 9, 14, 17)])
def test_maxfilter_amax_matches_numpy_chain(region):
    """The FP8 calibration statistic (per-channel maximum after the first and after the second
    max-filter, over the whole padded extent the layers compute) equals an independent numpy
    evaluation: row m of the result is the m-th max-filter and column c its channel c. Pins the
    layer chain (the second maxima depend on the first max-filter's output) and the m * C + c
    indexing, for the whole slice and for a region with true context."""
    params = teacher_params()
    sl = synth.em_volume(synth.BASE_SEED + 11, 1, 26, 31)[0]
    y0, x0, h, w = region if region else (0, 0, 26, 31)
    got = oracle.maxfilter_amax(T, params, sl, y0, x0, h, w)
    m1, m2 = _numpy_teacher_maxfilter_maps(params, sl, y0, x0, h, w)
    assert got.shape == (2, 32)
    assert m1.shape[1:] == (h + 9, w + 9) and m2.shape[1:] == (h + 4, w + 4)
    np.testing.assert_allclose(got[0], m1.reshape(32, -1).max(axis=1), rtol=1e-12, atol=0)
    np.testing.assert_allclose(got[1], m2.reshape(32, -1).max(axis=1), rtol=1e-12, atol=0)
    # the channels differ from one another, so a permuted or transposed result would not pass
    assert np.unique(np.round(got, 9)).size >= 40


def test_truth_head_fixture_is_a_membrane_classifier():
    """The second teacher workload's head (tests/golden/truth_head.json) recovers the generator's
    own membrane flag on a slice it was not fitted or selected on: well above the 82 % that a
    constant 'no membrane' answer scores, with about the true membrane fraction marked; and its
    regularisation strength follows the stated rule from the recorded held-out accuracies."""
    import json
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from _common import truth_head_teacher_params
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "truth_head.json")) as f:
        fx = json.load(f)
    accs = {float(k): v for k, v in fx["held_out_accuracy_by_lambda"].items()}
    best = max(accs.values())
    assert fx["lambda"] == max(lam for lam, a in accs.items() if a >= best - 1e-3)
    p = truth_head_teacher_params()
    s, truth = synth.em_slice_truth(synth.slice_seed(synth.BASE_SEED + 23, 0, 0), 192, 192)
    prob = oracle.forward_region(T, p, s)
    acc = ((prob >= 0.5) == (truth > 0)).mean()
    assert acc >= 0.95, acc
    assert abs((prob >= 0.5).mean() - truth.mean()) < 0.03
    # the map straddles the decision threshold: confident on most pixels, ambiguous on a few
    assert ((prob >= 0.3) & (prob <= 0.7)).mean() < 0.1 and (prob < 0.05).mean() > 0.5
