"""Pins of the post-filter oracle (Section 2, post-processing) against facts that
do not come from the oracle: a library cross-correlation, the identity of a
filter whose last layer is zero, and a filter of delta kernels whose output
follows by hand."""
import numpy as np
import pytest

import lf_inputs
import oracle

signal = pytest.importorskip("scipy.signal")

N_WEIGHTS = 3347


def test_weight_layout_has_the_declared_size():
    assert sum(int(np.prod(s)) for s in oracle.POST_SHAPES) == N_WEIGHTS


def test_conv3x3_equals_library_cross_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 13, 9))
    W = rng.standard_normal((5, 4, 3, 3))
    b = rng.standard_normal(5)
    got = oracle.conv3x3(x, W, b)
    for o in range(5):
        want = b[o] + sum(signal.correlate2d(x[i], W[o, i], mode="same", boundary="fill", fillvalue=0.0)
                          for i in range(4))
        np.testing.assert_allclose(got[o], want, rtol=0, atol=1e-12)


def _weights(W1=None, b1=None, W2=None, b2=None, W3=None, b3=None):
    parts = [W1, b1, W2, b2, W3, b3]
    return np.concatenate([np.zeros(int(np.prod(s))) if p is None else np.asarray(p, float).reshape(-1)
                           for p, s in zip(parts, oracle.POST_SHAPES)])


def test_zero_last_layer_is_the_identity_on_hit_pixels():
    rng = np.random.default_rng(2)
    w = _weights(W1=rng.standard_normal((16, 4, 3, 3)), b1=rng.standard_normal(16),
                 W2=rng.standard_normal((16, 16, 3, 3)), b2=rng.standard_normal(16))
    f = rng.uniform(0, 1, (4, 11, 17))
    f[3] = rng.uniform(0, 1, (11, 17)) < 0.6
    out = oracle.post_filter(w, f)
    np.testing.assert_array_equal(out, f[:3] * f[3])


def test_delta_kernels_scale_the_colour():
    # hidden channel c copies input channel c (c < 4) through two ReLU layers of centre
    # taps; the last layer adds half of channels 0..2: out = 1.5 RGB on hit pixels
    W1 = np.zeros((16, 4, 3, 3))
    W2 = np.zeros((16, 16, 3, 3))
    W3 = np.zeros((3, 16, 3, 3))
    for c in range(4):
        W1[c, c, 1, 1] = 1.0
        W2[c, c, 1, 1] = 1.0
    for c in range(3):
        W3[c, c, 1, 1] = 0.5
    rng = np.random.default_rng(3)
    f = rng.uniform(0, 1, (4, 8, 12))
    f[3] = 1.0
    f[3, 2:4, 5:9] = 0.0
    out = oracle.post_filter(_weights(W1=W1, W2=W2, W3=W3), f)
    np.testing.assert_allclose(out, 1.5 * f[:3] * f[3], rtol=0, atol=1e-15)


def test_a_shifted_kernel_moves_the_image():
    # W1 takes channel 0 from the pixel to the right (dx = 2), W2 and W3 centre taps:
    # out_R(y, x) = R(y, x) + R(y, x + 1), zero past the right edge
    W1 = np.zeros((16, 4, 3, 3))
    W2 = np.zeros((16, 16, 3, 3))
    W3 = np.zeros((3, 16, 3, 3))
    W1[0, 0, 1, 2] = 1.0
    W2[0, 0, 1, 1] = 1.0
    W3[0, 0, 1, 1] = 1.0
    rng = np.random.default_rng(4)
    f = rng.uniform(0, 1, (4, 6, 7))
    f[3] = 1.0
    out = oracle.post_filter(_weights(W1=W1, W2=W2, W3=W3), f)
    want = f[0].copy()
    want[:, :-1] += f[0][:, 1:]
    np.testing.assert_allclose(out[0], want, rtol=0, atol=1e-15)
    np.testing.assert_allclose(out[1:], f[1:3], rtol=0, atol=1e-15)


def test_features_mark_the_pixels_whose_ray_meets_the_sphere():
    v = lf_inputs.look_at((2.5, 0.3, 0.2), (0, 0, 0), 20, 14)
    img = np.ones((v.pixels, 4))
    f = oracle.post_features(v, img)
    hits = sum(oracle.trace_pixel(1.0, (0, 0, 0), v, x, y)[0] for y in range(14) for x in range(20))
    assert f[3].sum() == hits and 0 < hits < v.pixels
    np.testing.assert_array_equal(f[:3], 1.0)
