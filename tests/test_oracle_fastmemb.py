"""Pins of the oracle's FastMemb dense form (Sec. 2.2, "A lightweight network architecture" and
"Accelerating dense computation") to facts outside the oracle: the printed field of view (53x53)
and parameter budget (about 70k), the patch calculation with real stride-2 max-pooling, a literal
max-pooling-fragments evaluation (k^2 sub-matrices per stride-2 op, recursed, interleaved after
the softmax), the dense-vs-sliding-window multiplication ratio (printed as 284x), and library
routines for the new primitives (dilated correlation, dilated max-filter, max-out, softmax).
CPU only."""
import numpy as np
import pytest
from numpy.lib.stride_tricks import sliding_window_view

import oracle
import synth
from test_oracle_pins import split_params

F = synth.FASTMEMB


def fm_params(seed=synth.FASTMEMB_WEIGHT_SEED):
    return synth.init_params(F, seed).astype(np.float64)


# --- independent numpy building blocks (sliding windows + einsum, not the oracle's loops) --------

def np_conv(x, W, b, stride_dil=1):
    """Valid cross-correlation, dilation d, via sliding windows."""
    k = W.shape[-1]
    span = (k - 1) * stride_dil + 1
    win = sliding_window_view(x, (span, span), axis=(1, 2))[..., ::stride_dil, ::stride_dil]
    return np.einsum("chwyx,ocyx->ohw", win, W) + b[:, None, None]


def np_maxout(x, G):
    c, h, w = x.shape
    return x.reshape(c // G, G, h, w).max(axis=1)


def np_maxpool2_stride2(x):
    """Max-pooling 2x2 with stride 2 (floor: a trailing odd row/column is dropped)."""
    c, h, w = x.shape
    h2, w2 = h // 2, w // 2
    return x[:, :2 * h2, :2 * w2].reshape(c, h2, 2, w2, 2).max(axis=(2, 4))


def np_softmax_class1(z):
    e = np.exp(z - z.max(axis=0, keepdims=True))
    return e[1] / e.sum(axis=0)


def patch_network(patch, params):
    """FastMemb as the paper's patch calculation: 53x53 patch -> three [conv4 -> max-out 2 ->
    2x2 max-pool stride 2] stages -> conv4 -> 2-class softmax; one output pixel."""
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = split_params(F, params)
    x = patch[None]
    for W, b in ((W1, b1), (W2, b2), (W3, b3)):
        x = np_maxpool2_stride2(np_maxout(np_conv(x, W, b), 2))
    z = np_conv(x, W4, b4)
    assert z.shape == (2, 1, 1)
    return float(np_softmax_class1(z)[0, 0])


# --- the architecture's printed figures -----------------------------------------------------------

def test_field_of_view_53_and_about_70k_parameters():
    assert oracle.net_radius(F) == 26                      # 53x53 field of view
    assert oracle.param_count(F) == synth.param_count(F) == 67778
    assert abs(67778 - 70000) / 70000 < 0.05               # "70k parameters"
    # without max-out the same layers would hold about half as many
    no_maxout = tuple(l[:6] + (1,) for l in F)
    assert oracle.param_count(no_maxout) < 35000


def test_patch_network_shapes_close_at_53():
    """Three conv4/pool2 stages and a conv4 map exactly a 53x53 patch to 1x1 (and 52 to 0)."""
    n = 53
    for _ in range(3):
        n = (n - 3) // 2
    assert n - 3 == 1
    n = 52
    for _ in range(3):
        n = (n - 3) // 2
    assert n - 3 < 1


def test_dense_to_sliding_window_multiplication_ratio():
    """Sliding-window FastMemb on each pixel's 53x53 patch against the dense form's per-pixel
    multiplications; the paper prints about 284x fewer for dense computation."""
    convs = [l for l in F if l[0] != synth.MAXFILTER]
    dense = sum(l[3] * l[6] * l[2] * l[1] * l[1] for l in convs)
    assert dense == 67584
    n, patch = 53, 0
    for l in convs:
        n = n - 3
        patch += n * n * l[3] * l[6] * l[2] * l[1] * l[1]
        n //= 2
    ratio = patch / dense
    assert 284 * 0.93 < ratio < 284 * 1.10, ratio


# --- the new primitives against library routines ---------------------------------------------------

@pytest.mark.parametrize("d", [1, 2, 3, 8])
def test_dilated_conv_matches_scipy_with_zero_inserted_kernel(d):
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(30 + d)
    x = rng.standard_normal((3, 40, 37))
    W = rng.standard_normal((4, 3, 4, 4))
    b = rng.standard_normal(4)
    Wd = np.zeros((4, 3, 3 * d + 1, 3 * d + 1))
    Wd[:, :, ::d, ::d] = W
    ref = np.stack([b[co] + sum(signal.correlate2d(x[ci], Wd[co, ci], mode="valid") for ci in range(3))
                    for co in range(4)])
    y = oracle.conv_dil(x, W, b, d, relu=False)
    assert y.shape == (4, 40 - 3 * d, 37 - 3 * d)
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("d", [1, 2, 4, 5])
def test_dilated_maxfilter_matches_sliding_window_max(d):
    rng = np.random.default_rng(40 + d)
    x = rng.standard_normal((2, 19, 23))
    win = sliding_window_view(x, (d + 1, d + 1), axis=(1, 2))[..., ::d, ::d]
    ref = win.max(axis=(-1, -2))
    np.testing.assert_array_equal(oracle.maxfilter2_dil(x, d), ref)


def test_maxout_groups_are_adjacent_channels():
    rng = np.random.default_rng(50)
    x = rng.standard_normal((12, 5, 7))
    for G in (1, 2, 3, 4):
        y = oracle.maxout(x, G)
        assert y.shape == (12 // G, 5, 7)
        for c in range(12 // G):
            np.testing.assert_array_equal(y[c], np.max(x[c * G:(c + 1) * G], axis=0))


def test_softmax_head_closed_form_and_class_swap():
    rng = np.random.default_rng(60)
    x = rng.standard_normal((1, 9, 11))
    W = rng.standard_normal((2, 1, 1, 1))
    b = rng.standard_normal(2)
    layers = ((synth.HEAD_SOFTMAX2, 1, 1, 2, 0, 1, 1),)
    prm = np.concatenate([W.ravel(), b])
    p = oracle.run_layers(layers, prm, x[0])
    z0 = W[0, 0, 0, 0] * x[0] + b[0]
    z1 = W[1, 0, 0, 0] * x[0] + b[1]
    np.testing.assert_allclose(p, np.exp(z1) / (np.exp(z0) + np.exp(z1)), rtol=0, atol=1e-15)
    swapped = np.concatenate([W[::-1].ravel(), b[::-1]])
    np.testing.assert_allclose(oracle.run_layers(layers, swapped, x[0]), 1.0 - p, rtol=0, atol=1e-15)


def test_maxout_with_dominated_second_group_equals_plain_network():
    """Group 1 of every max-out pair = group 0 minus 10 in the bias: the max always picks group 0,
    so the network equals the G=1 network of the group-0 filters (fixes the channel order c*G+g)."""
    prm = fm_params()
    parts = split_params(F, prm)
    plain_layers = tuple(l[:6] + (1,) for l in F)
    plain, mod = [], []
    for (W, b), l in zip(parts, [l for l in F if l[0] != synth.MAXFILTER]):
        G = l[6]
        if G == 1:
            plain += [W.ravel(), b]
            mod += [W.ravel(), b]
            continue
        W0, b0 = W[0::G], b[0::G]
        Wm, bm = W.copy(), b.copy()
        Wm[1::G] = W0
        bm[1::G] = b0 - 10.0
        plain += [W0.ravel(), b0]
        mod += [Wm.ravel(), bm]
    s = synth.em_slice(7001, 64, 60)
    a = oracle.forward_region(F, np.concatenate(mod), s)
    c = oracle.forward_region(plain_layers, np.concatenate(plain), s)
    np.testing.assert_array_equal(a, c)


# --- dense form against the patch calculation and the max-pooling fragments ------------------------

def test_dense_equals_patch_calculation_with_stride2_pooling():
    prm = fm_params()
    s = synth.em_slice(7002, 70, 66)
    dense = oracle.forward_region(F, prm, s)
    assert dense.shape == s.shape
    padded = np.pad(s.astype(np.float64) / 255.0, 26, mode="reflect")
    rng = np.random.default_rng(70)
    pix = [(0, 0), (69, 65), (0, 65), (69, 0), (26, 26), (35, 3)]
    pix += [tuple(int(v) for v in rng.integers(0, (70, 66))) for _ in range(10)]
    for i, j in pix:
        p = patch_network(padded[i:i + 53, j:j + 53], prm)
        assert abs(p - dense[i, j]) < 1e-12, (i, j, p, dense[i, j])
        assert abs(oracle.patch_pixel(F, prm, s, i, j) - dense[i, j]) < 1e-12


def fragments_forward(xp, params):
    """Max-pooling fragments, generalised: every stride-2 pooling is a stride-1 2x2 max-filter
    followed by 2-factor sub-sampling at the 4 offsets, giving 4 independent sub-matrices that
    the later layers process separately (as plain, non-dilated layers). After the softmax the
    sub-matrices are interleaved back into the dense map. Each fragment carries its origin and
    step in the dense output frame."""
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = split_params(F, params)
    frags = [(0, 0, 1, xp[None])]
    for W, b in ((W1, b1), (W2, b2), (W3, b3)):
        nxt = []
        for oy, ox, step, x in frags:
            m = np_maxout(np_conv(x, W, b), 2)
            m = np.maximum(np.maximum(m[:, :-1, :-1], m[:, 1:, :-1]), np.maximum(m[:, :-1, 1:], m[:, 1:, 1:]))
            for sy in (0, 1):
                for sx in (0, 1):
                    nxt.append((oy + step * sy, ox + step * sx, 2 * step, m[:, sy::2, sx::2]))
        frags = nxt
    assert len(frags) == 64
    H, W = xp.shape[0] - 52, xp.shape[1] - 52
    out = np.full((H, W), np.nan)
    for oy, ox, step, x in frags:
        p = np_softmax_class1(np_conv(x, W4, b4))
        h, w = p.shape
        assert step == 8
        ys, xs = np.arange(h) * step + oy, np.arange(w) * step + ox
        keep_y, keep_x = ys < H, xs < W
        out[np.ix_(ys[keep_y], xs[keep_x])] = p[np.ix_(keep_y, keep_x)]
    return out


def test_dense_equals_max_pooling_fragments_interleaved():
    prm = fm_params(synth.FASTMEMB_WEIGHT_SEED + 3)
    s = synth.em_slice(7003, 45, 38)
    dense = oracle.forward_region(F, prm, s)
    frag = fragments_forward(np.pad(s.astype(np.float64) / 255.0, 26, mode="reflect"), prm)
    assert not np.isnan(frag).any()
    np.testing.assert_allclose(dense, frag, rtol=0, atol=1e-12)


def test_fastmemb_output_is_a_probability_map_and_needs_27_pixels():
    prm = fm_params()
    p = oracle.forward_region(F, prm, synth.em_slice(7004, 27, 27))
    assert p.shape == (27, 27) and np.all((p >= 0) & (p <= 1))
    with pytest.raises(RuntimeError):
        oracle.forward_region(F, prm, synth.em_slice(7004, 26, 40))


def pruned_fragments_forward(xp, params):
    """The fragment tree pruned at the first stride-2 pool to its offset (0, 0) branch: 16 of the 64
    fragments, interleaved after the softmax, give the dense map at even rows and columns."""
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = split_params(F, params)
    m = np_maxout(np_conv(xp[None], W1, b1), 2)
    m = np.maximum(np.maximum(m[:, :-1, :-1], m[:, 1:, :-1]), np.maximum(m[:, :-1, 1:], m[:, 1:, 1:]))
    frags = [(0, 0, 2, m[:, 0::2, 0::2])]
    for W, b in ((W2, b2), (W3, b3)):
        nxt = []
        for oy, ox, step, x in frags:
            m = np_maxout(np_conv(x, W, b), 2)
            m = np.maximum(np.maximum(m[:, :-1, :-1], m[:, 1:, :-1]), np.maximum(m[:, :-1, 1:], m[:, 1:, 1:]))
            for sy in (0, 1):
                for sx in (0, 1):
                    nxt.append((oy + step * sy, ox + step * sx, 2 * step, m[:, sy::2, sx::2]))
        frags = nxt
    assert len(frags) == 16
    H, W = xp.shape[0] - 52, xp.shape[1] - 52
    out = np.full(((H + 1) // 2, (W + 1) // 2), np.nan)
    for oy, ox, step, x in frags:
        p = np_softmax_class1(np_conv(x, W4, b4))
        ys, xs = np.arange(p.shape[0]) * step + oy, np.arange(p.shape[1]) * step + ox
        ky, kx = ys < H, xs < W
        out[np.ix_(ys[ky] // 2, xs[kx] // 2)] = p[np.ix_(ky, kx)]
    return out


@pytest.mark.parametrize("shape", [(44, 38), (45, 37)])
def test_subsampled_output_is_the_pruned_fragment_tree(shape):
    """Sec. 2.2 (Fig. 3a caption): pruning the recursion tree sub-samples the output. The branch of
    the first pool's offset (0, 0) equals the dense map at even positions."""
    prm = fm_params(synth.FASTMEMB_WEIGHT_SEED + 4)
    s = synth.em_slice(7005, *shape)
    dense = oracle.forward_region(F, prm, s)
    pruned = pruned_fragments_forward(np.pad(s.astype(np.float64) / 255.0, 26, mode="reflect"), prm)
    assert not np.isnan(pruned).any() and pruned.shape == dense[::2, ::2].shape
    np.testing.assert_allclose(pruned, dense[::2, ::2], rtol=0, atol=1e-12)


# ---- FastMemb_3nm (Sec. 2.2, "A subsampling CNN for 3 nm data") ------------------------------------

F3 = synth.FASTMEMB_3NM


def test_fastmemb_3nm_field_of_view_parameters_and_flop_ratio():
    """One more conv/pool pair: field of view 109 by the arithmetic of the architecture, the value
    Sec. 3.2 prints for the same four-pair structure (this section prints 105); 100,610
    parameters; 4x the pixels at 100,352 vs 67,584 multiplications per pixel = 5.94x the FLOPs
    of FastMemb_6nm, against the printed 5.86x (text, "486 % more") and 5.68x (table)."""
    assert oracle.net_radius(F3) == 54
    assert oracle.param_count(F3) == synth.param_count(F3) == 100610
    per_px = lambda layers: sum(l[3] * l[6] * l[2] * l[1] ** 2 for l in layers if l[0] != synth.MAXFILTER)
    assert per_px(F) == 67584 and per_px(F3) == 100352
    ratio = 4 * per_px(F3) / per_px(F)
    assert abs(ratio - 5.86) / 5.86 < 0.02 and abs(ratio - 5.68) / 5.68 < 0.05, ratio
    n = 109
    for _ in range(4):
        n = (n - 3) // 2
    assert n - 3 == 1


def test_fastmemb_3nm_dense_equals_patch_calculation():
    prm = synth.init_params(F3, synth.FASTMEMB_3NM_WEIGHT_SEED).astype(np.float64)
    parts = split_params(F3, prm)
    s = synth.em_slice(7006, 70, 64)
    dense = oracle.forward_region(F3, prm, s)
    padded = np.pad(s.astype(np.float64) / 255.0, 54, mode="reflect")
    rng = np.random.default_rng(80)
    pix = [(0, 0), (69, 63), (0, 63), (35, 31)] + [tuple(int(v) for v in rng.integers(0, (70, 64))) for _ in range(6)]
    for i, j in pix:
        x = padded[i:i + 109, j:j + 109][None]
        for W, b in parts[:-1]:
            x = np_maxpool2_stride2(np_maxout(np_conv(x, W, b), 2))
        z = np_conv(x, *parts[-1])
        assert z.shape == (2, 1, 1)
        assert abs(float(np_softmax_class1(z)[0, 0]) - dense[i, j]) < 1e-12
