"""Pins of the FP64 CNN reference (oracle/cnn.py): the convolution equals
scipy's N-D correlation with zero padding, pooling/upsampling backward passes
are the adjoints of the forward passes, and every gradient (layer and whole
encoder-decoder) matches central finite differences."""
import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import cnn


def test_conv3d_equals_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 5, 6, 4))
    W = rng.standard_normal((2, 3, 27))
    b = rng.standard_normal(2)
    y = cnn.conv3d(x, W, b)
    for o in range(2):
        ref = b[o] + sum(ndi.correlate(x[c], W[o, c].reshape(3, 3, 3), mode="constant", cval=0.0) for c in range(3))
        np.testing.assert_allclose(y[o], ref, atol=1e-12)


def test_pool_and_upsample_backward_are_adjoints():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((2, 4, 6, 8))
    s = rng.standard_normal((2, 2, 3, 4))
    assert abs(np.sum(cnn.avgpool2(a) * s) - np.sum(a * cnn.avgpool2_backward(s))) < 1e-12
    assert abs(np.sum(cnn.upsample2(s) * a) - np.sum(s * cnn.upsample2_backward(a))) < 1e-12


def test_conv3d_backward_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 3, 4, 3))
    W = rng.standard_normal((3, 2, 27))
    b = rng.standard_normal(3)
    gy = rng.standard_normal((3, 3, 4, 3))
    dx, dW, db = cnn.conv3d_backward(x, W, gy)
    f = lambda x_, W_, b_: np.sum(gy * cnn.conv3d(x_, W_, b_))  # noqa: E731
    eps = 1e-6
    for arr, grad in ((x, dx), (W, dW), (b, db)):
        for _ in range(6):
            idx = tuple(rng.integers(s) for s in arr.shape)
            old = arr[idx]
            arr[idx] = old + eps
            fp = f(x, W, b)
            arr[idx] = old - eps
            fm = f(x, W, b)
            arr[idx] = old
            assert abs((fp - fm) / (2 * eps) - grad[idx]) < 1e-6


def test_unet_gradient_directional_derivative():
    """d/de sum(gy * unet(x; theta + e v)) at e = 0 equals <grad, v>."""
    rng = np.random.default_rng(3)
    widths = (4, 6, 8, 10)
    params = cnn.unet_init(3, 2, seed=5, widths=widths)
    for k in params:  # make every layer active and non-trivial
        W, b = params[k]
        params[k] = (W * 3.0, rng.standard_normal(b.shape) * 0.1)
    x = rng.standard_normal((3, 8, 8, 8))
    y, cache = cnn.unet_forward(params, x)
    assert y.shape == (2, 8, 8, 8)
    gy = rng.standard_normal(y.shape)
    grads = cnn.unet_backward(params, cache, gy)
    v = {k: (rng.standard_normal(W.shape), rng.standard_normal(b.shape)) for k, (W, b) in params.items()}
    pred = sum(np.sum(grads[k][0] * v[k][0]) + np.sum(grads[k][1] * v[k][1]) for k in params)
    eps = 1e-6

    def f(e):
        p = {k: (W + e * v[k][0], b + e * v[k][1]) for k, (W, b) in params.items()}
        return np.sum(gy * cnn.unet_forward(p, x)[0])
    fd = (f(eps) - f(-eps)) / (2 * eps)
    assert abs(fd - pred) <= 1e-6 * max(1.0, abs(pred))


@pytest.mark.parametrize("name", ["e0a", "e3b", "d1", "out"])
def test_unet_layer_gradients_one_entry(name):
    rng = np.random.default_rng(4)
    params = cnn.unet_init(2, 2, seed=1, widths=(3, 4, 5, 6))
    x = rng.standard_normal((2, 8, 8, 8))
    y, cache = cnn.unet_forward(params, x)
    gy = rng.standard_normal(y.shape)
    g = cnn.unet_backward(params, cache, gy)[name][0]
    W = params[name][0]
    idx = tuple(rng.integers(s) for s in W.shape)
    eps = 1e-6
    old = W[idx]
    W[idx] = old + eps
    fp = np.sum(gy * cnn.unet_forward(params, x)[0])
    W[idx] = old - eps
    fm = np.sum(gy * cnn.unet_forward(params, x)[0])
    W[idx] = old
    assert abs((fp - fm) / (2 * eps) - g[idx]) <= 1e-6 * max(1.0, abs(g[idx]))
