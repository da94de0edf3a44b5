"""FP64 CPU reference of the convolutional network used as a learned
preconditioner: the layers, their gradients, and the encoder-decoder.

TEST INFRASTRUCTURE ONLY (part of the FP64 CPU oracle; see oracle/__init__.py).

The paper has no network; the learned preconditioner is an extension (a
3D convolutional encoder-decoder mapping a residual, together with the
medium, to a correction of the iterate).  This module is the plain,
slow definition the GPU training and inference kernels are checked
against: every layer is written from its mathematical definition.

Tensors are float64 arrays (C, Z, Y, X) (one sample).  Convolutions are
3x3x3, stride 1, zero padding 1 ("same"): out[o, p] = b[o] + sum_{c, t}
W[o, c, t] in[c, p + t], t in {-1, 0, 1}^3 with taps ordered t = (dz, dy, dx)
-> index (dz+1)*9 + (dy+1)*3 + (dx+1).
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shift(a: np.ndarray, t) -> np.ndarray:
    """s[c, p] = a[c, p + t] with zeros outside."""
    dz, dy, dx = t
    C, Z, Y, X = a.shape
    out = np.zeros_like(a)
    zs = slice(max(0, -dz), min(Z, Z - dz))
    ys = slice(max(0, -dy), min(Y, Y - dy))
    xs = slice(max(0, -dx), min(X, X - dx))
    zi = slice(max(0, dz), min(Z, Z + dz))
    yi = slice(max(0, dy), min(Y, Y + dy))
    xi = slice(max(0, dx), min(X, X + dx))
    out[:, zs, ys, xs] = a[:, zi, yi, xi]
    return out


def conv3d(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """W: (Cout, Cin, 27), b: (Cout,)."""
    out = np.zeros((W.shape[0],) + x.shape[1:])
    for ti, t in enumerate(TAPS):
        out += np.einsum("oc,czyx->ozyx", W[:, :, ti], _shift(x, t))
    return out + b[:, None, None, None]


def conv3d_backward(x: np.ndarray, W: np.ndarray, gy: np.ndarray):
    """Gradients (dx, dW, db) of sum(gy * conv3d(x, W, b))."""
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for ti, t in enumerate(TAPS):
        xs = _shift(x, t)
        dW[:, :, ti] = np.einsum("ozyx,czyx->oc", gy, xs)
        # d/dx of in[c, p + t]: scatter back by -t
        dx += _shift(np.einsum("oc,ozyx->czyx", W[:, :, ti], gy), tuple(-v for v in t))
    db = gy.sum(axis=(1, 2, 3))
    return dx, dW, db


def relu(x):
    return np.maximum(x, 0.0)


def relu_backward(x, gy):
    return gy * (x > 0)


def avgpool2(x: np.ndarray) -> np.ndarray:
    """Mean over 2x2x2 blocks (even sizes)."""
    C, Z, Y, X = x.shape
    return x.reshape(C, Z // 2, 2, Y // 2, 2, X // 2, 2).mean(axis=(2, 4, 6))


def avgpool2_backward(gy: np.ndarray) -> np.ndarray:
    return np.repeat(np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def upsample2(x: np.ndarray) -> np.ndarray:
    """Nearest-neighbour 2x upsampling."""
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def upsample2_backward(gy: np.ndarray) -> np.ndarray:
    C, Z, Y, X = gy.shape
    return gy.reshape(C, Z // 2, 2, Y // 2, 2, X // 2, 2).sum(axis=(2, 4, 6))


# --- the encoder-decoder ----------------------------------------------------

def unet_layers(c_in: int, c_out: int, widths=(16, 32, 48, 64)):
    """(name, Cin, Cout) of every convolution, in execution order."""
    c0, c1, c2, c3 = widths
    return [("e0a", c_in, c0), ("e0b", c0, c0), ("e1a", c0, c1), ("e1b", c1, c1),
            ("e2a", c1, c2), ("e2b", c2, c2), ("e3a", c2, c3), ("e3b", c3, c3),
            ("d2", c3 + c2, c2), ("d1", c2 + c1, c1), ("d0", c1 + c0, c0), ("out", c0, c_out)]


def unet_init(c_in: int, c_out: int, seed: int, widths=(16, 32, 48, 64)):
    """He-style initial weights (FP64), last layer scaled down."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = {}
    for name, ci, co in unet_layers(c_in, c_out, widths):
        std = np.sqrt(2.0 / (27 * ci)) * (0.1 if name == "out" else 1.0)
        params[name] = (rng.standard_normal((co, ci, 27)) * std, np.zeros(co))
    return params


def _keep(a):
    return a


def unet_forward(params, x: np.ndarray, store=None):
    """Returns (output, cache of intermediate activations for the backward).

    `store` (default: exact) is applied wherever an implementation keeps an
    intermediate tensor in memory (every layer output, pooled tensor); tests
    pass a rounding to a storage precision to model reduced-precision
    storage with exact arithmetic in between.
    """
    st = store or _keep
    c = {}

    def conv(name, inp, act=True):
        W, b = params[name]
        pre = conv3d(inp, W, b)
        c[name] = (inp, pre)
        return st(relu(pre)) if act else st(pre)

    s0 = conv("e0b", conv("e0a", st(x)))
    s1 = conv("e1b", conv("e1a", st(avgpool2(s0))))
    s2 = conv("e2b", conv("e2a", st(avgpool2(s1))))
    bt = conv("e3b", conv("e3a", st(avgpool2(s2))))
    d2 = conv("d2", np.concatenate([upsample2(bt), s2]))
    d1 = conv("d1", np.concatenate([upsample2(d2), s1]))
    d0 = conv("d0", np.concatenate([upsample2(d1), s0]))
    y = conv("out", d0, act=False)
    return y, c


def unet_backward(params, cache, gy: np.ndarray, store=None):
    """Gradients {name: (dW, db)} of sum(gy * unet(x)); `store` as in
    unet_forward, applied to every stored gradient tensor."""
    st = store or _keep
    grads = {}

    def back(name, g, act=True):
        inp, pre = cache[name]
        if act:
            g = relu_backward(pre, g)
        dx, dW, db = conv3d_backward(inp, params[name][0], g)
        grads[name] = (dW, db)
        return st(dx)

    g_d0 = back("out", st(gy), act=False)
    g = back("d0", g_d0)
    c1 = params["d1"][0].shape[0]
    g_up1, g_s0 = g[:c1], g[c1:]
    g = back("d1", st(upsample2_backward(g_up1)))
    c2 = params["d2"][0].shape[0]
    g_up2, g_s1 = g[:c2], g[c2:]
    g = back("d2", st(upsample2_backward(g_up2)))
    c3 = params["e3b"][0].shape[0]
    g_up3, g_s2 = g[:c3], g[c3:]
    g = back("e3a", back("e3b", st(upsample2_backward(g_up3))))
    g = back("e2a", back("e2b", st(avgpool2_backward(g) + g_s2)))
    g = back("e1a", back("e1b", st(avgpool2_backward(g) + g_s1)))
    back("e0a", back("e0b", st(avgpool2_backward(g) + g_s0)))
    return grads
