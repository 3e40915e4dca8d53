"""Plain FP64 reference of the layers of the learned start-model network.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the CNN kernels of the
library are checked against these functions; nothing in the product imports
them. The network is not from the paper (whose Limitations section names the
starting model of FWI as its weak point); the layers are textbook definitions,
written out directly with numpy:

* conv2d: cross-correlation with a 3x3 kernel, zero padding 1, stride (sh, sw):
  y[o, b, i, j] = bias[o] + sum_{c, p, q} w[o, c, p, q] x[c, b, sh i + p - 1, sw j + q - 1];
  activations are laid out channel-major, [C][B][H][W].
* its two gradients: dx by scattering dy back through the same index map, dw and
  dbias by correlating dy with x;
* ReLU and its gradient (mask y > 0);
* nearest-neighbour upsampling by 2 in both axes and its gradient (2x2 sums);
* the mean squared error L = 1/(2 n) sum (p - t)^2 and dL/dp = (p - t) / n;
* one Adam step (Kingma & Ba), bias-corrected.

Every function takes and returns FP64 (or complex128, for complex-step checks)
numpy arrays.
"""

from __future__ import annotations

import numpy as np


def conv_out(n: int, s: int) -> int:
    """Output length of a 3-tap, pad-1, stride-s axis of length n."""
    return (n - 1) // s + 1


def conv2d(x, w, bias, sh, sw):
    """x [C][B][H][W], w [O][C][3][3], bias [O] -> y [O][B][Ho][Wo]."""
    C, B, H, W = x.shape
    O = w.shape[0]
    Ho, Wo = conv_out(H, sh), conv_out(W, sw)
    xp = np.zeros((C, B, H + 2, W + 2), dtype=np.result_type(x, w))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    y = np.zeros((O, B, Ho, Wo), dtype=xp.dtype)
    for p in range(3):
        for q in range(3):
            patch = xp[:, :, p:p + sh * (Ho - 1) + 1:sh, q:q + sw * (Wo - 1) + 1:sw]  # [C][B][Ho][Wo]
            y += np.einsum("oc,cbij->obij", w[:, :, p, q], patch)
    return y + np.asarray(bias)[:, None, None, None]


def conv2d_backward(x, w, dy, sh, sw):
    """Gradients (dx, dw, dbias) of sum(dy * conv2d(x, w, bias))."""
    C, B, H, W = x.shape
    O, _, Ho, Wo = dy.shape[0], None, dy.shape[2], dy.shape[3]
    xp = np.zeros((C, B, H + 2, W + 2), dtype=np.result_type(x, w, dy))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros(w.shape, dtype=xp.dtype)
    for p in range(3):
        for q in range(3):
            sl = (slice(None), slice(None), slice(p, p + sh * (Ho - 1) + 1, sh), slice(q, q + sw * (Wo - 1) + 1, sw))
            dw[:, :, p, q] = np.einsum("obij,cbij->oc", dy, xp[sl])
            dxp[sl] += np.einsum("oc,obij->cbij", w[:, :, p, q], dy)
    return dxp[:, :, 1:H + 1, 1:W + 1], dw, dy.sum(axis=(1, 2, 3))


def relu(y):
    return np.where(y.real > 0, y, 0)


def relu_backward(y, dy):
    """dL/d(pre-activation) from the post-activation y and dL/dy."""
    return np.where(y.real > 0, dy, 0)


def upsample2(x):
    """Nearest-neighbour 2x upsampling of the last two axes."""
    return np.repeat(np.repeat(x, 2, axis=-2), 2, axis=-1)


def upsample2_backward(dy):
    C, B, H2, W2 = dy.shape
    return dy.reshape(C, B, H2 // 2, 2, W2 // 2, 2).sum(axis=(3, 5))


def mse(p, t):
    """L = 1/(2n) sum (p - t)^2 and dL/dp."""
    r = p - t
    n = r.size
    return 0.5 * np.sum(r * r) / n, r / n


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(x):
    """FP32 values rounded to the nearest BF16 (8-bit significand, ties to even),
    returned as float64: the operands the tensor-core GEMMs actually multiply."""
    a = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (a >> 16) & 1
    r = ((a + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
