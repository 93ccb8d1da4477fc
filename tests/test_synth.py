"""The seeded input generator: determinism, shapes and the statistics of its recipe."""
import numpy as np

import synth


def test_slice_is_deterministic_and_seed_dependent():
    a = synth.em_slice(42, 64, 80)
    b = synth.em_slice(42, 64, 80)
    c = synth.em_slice(43, 64, 80)
    assert a.shape == (64, 80) and a.dtype == np.uint8
    np.testing.assert_array_equal(a, b)
    assert (a != c).any()


def test_default_density_is_120_cells_per_256_squared():
    assert synth.default_cells(256, 256) == 120
    assert synth.default_cells(1024, 1024) == 1920
    assert synth.default_cells(4096, 4096) == 30720


def test_intensity_statistics():
    s = synth.em_slice(synth.slice_seed(synth.BASE_SEED, 0, 0), 256, 256)
    dark = s < 115
    # membranes (2-3 px wide) cover a minority of pixels; interiors are bright
    assert 0.08 < dark.mean() < 0.35
    assert 150 < s[~dark].mean() < 185
    assert 40 < s[dark].mean() < 110


def test_volume_slices_use_slice_seeds():
    v = synth.em_volume(7, 3, 32, 40, block=2)
    for z in range(3):
        np.testing.assert_array_equal(v[z], synth.em_slice(synth.slice_seed(7, 2, z), 32, 40))


def test_he_normal_scale():
    w, b = synth.he_normal(5, 800, 25600, 32, 0.01)
    assert abs(w.std() - np.sqrt(2 / 800)) < 0.002
    assert abs(w.mean()) < 0.002
    assert b.std() < 0.02
    w0, b0 = synth.he_normal(5, 800, 10, 4, 0.0)
    assert (b0 == 0).all()


def test_block_shapes_ranges():
    shapes = synth.block_shapes(9, 64)
    assert len(shapes) == 64
    for d, h, w in shapes:
        assert 1 <= d <= 16 and 256 <= h <= 1536 and 256 <= w <= 1536
    assert synth.block_shapes(9, 64) == shapes


def test_centred_head_has_zero_channel_mean_and_leaves_other_layers():
    a = synth.init_params(synth.FASTMEMB_3NM, 5)
    b = synth.init_params(synth.FASTMEMB_3NM, 5, center_head=True)
    n_head = 2 * 32 * 16 + 2
    np.testing.assert_array_equal(a[:-n_head], b[:-n_head])
    np.testing.assert_array_equal(a[-2:], b[-2:])
    w = b[-n_head:-2].reshape(2, 32, 16).astype(np.float64)
    assert np.abs(w.mean(axis=1)).max() < 1e-6


def test_centred_input_init_only_moves_first_layer_biases():
    a = synth.init_params(synth.STUDENT, synth.STUDENT_WEIGHT_SEED, bias_std=0.0)
    b = synth.init_params(synth.STUDENT, synth.STUDENT_WEIGHT_SEED, bias_std=0.0, centred_input=True)
    np.testing.assert_array_equal(a[:144], b[:144])
    np.testing.assert_array_equal(a[160:], b[160:])
    np.testing.assert_allclose(b[144:160], -0.5 * a[:144].reshape(16, 9).astype(np.float64).sum(axis=1), rtol=1e-6)
