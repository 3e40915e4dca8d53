"""Pins of the FP64 reference layers of the start-model network (oracle/cnn.py).

* conv2d against scipy.signal.correlate2d (a library routine written
  independently) channel by channel, for unit and non-unit strides;
* its backward against complex-step directional derivatives of the forward
  (the backward is written as a scatter, the forward as a gather);
* upsampling and its backward through the adjoint identity <U x, y> = <x, U^T y>;
* the MSE gradient against complex step; one Adam step against the update
  written out by hand for a scalar.
"""

import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn


def _rand(rng, *shape):
    return rng.standard_normal(shape)


@pytest.mark.parametrize("sh,sw", [(1, 1), (2, 1), (4, 2), (3, 3)])
def test_conv2d_equals_correlate2d(sh, sw):
    rng = np.random.default_rng(1 + sh + 10 * sw)
    C, B, H, W, O = 3, 2, 11, 9, 4
    x, w, b = _rand(rng, C, B, H, W), _rand(rng, O, C, 3, 3), _rand(rng, O)
    y = cnn.conv2d(x, w, b, sh, sw)
    assert y.shape == (O, B, cnn.conv_out(H, sh), cnn.conv_out(W, sw))
    for o in range(O):
        for bb in range(B):
            full = sum(correlate2d(np.pad(x[c, bb], 1), w[o, c], mode="valid") for c in range(C)) + b[o]
            np.testing.assert_allclose(y[o, bb], full[::sh, ::sw], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("sh,sw", [(1, 1), (2, 2), (4, 1)])
def test_conv2d_backward_vs_complex_step(sh, sw):
    rng = np.random.default_rng(7 * sh + sw)
    C, B, H, W, O = 2, 3, 10, 7, 3
    x, w, b = _rand(rng, C, B, H, W), _rand(rng, O, C, 3, 3), _rand(rng, O)
    dy = _rand(rng, O, B, cnn.conv_out(H, sh), cnn.conv_out(W, sw))
    dx, dw, db = cnn.conv2d_backward(x, w, dy, sh, sw)
    h = 1e-30
    L = lambda xx, ww, bb: np.sum(dy * cnn.conv2d(xx, ww, bb, sh, sw))
    for _ in range(3):
        ex, ew, eb = _rand(rng, *x.shape), _rand(rng, *w.shape), _rand(rng, *b.shape)
        assert np.sum(dx * ex) == pytest.approx(L(x + 1j * h * ex, w, b).imag / h, rel=1e-12)
        assert np.sum(dw * ew) == pytest.approx(L(x, w + 1j * h * ew, b).imag / h, rel=1e-12)
        assert np.sum(db * eb) == pytest.approx(L(x, w, b + 1j * h * eb).imag / h, rel=1e-12)


def test_relu_backward_masks_by_output():
    y = np.array([[-1.0, 0.0, 2.0]])
    np.testing.assert_array_equal(cnn.relu(y), [[0.0, 0.0, 2.0]])
    np.testing.assert_array_equal(cnn.relu_backward(cnn.relu(y), np.ones((1, 3))), [[0.0, 0.0, 1.0]])


def test_upsample_adjoint_identity():
    rng = np.random.default_rng(3)
    x = _rand(rng, 2, 3, 5, 4)
    u = cnn.upsample2(x)
    assert u.shape == (2, 3, 10, 8) and np.array_equal(u[:, :, 1::2, ::2], x)
    y = _rand(rng, *u.shape)
    assert np.sum(u * y) == pytest.approx(np.sum(x * cnn.upsample2_backward(y)), rel=1e-13)


def test_mse_gradient_vs_complex_step():
    rng = np.random.default_rng(4)
    p, t = _rand(rng, 5, 6), _rand(rng, 5, 6)
    L, g = cnn.mse(p, t)
    assert L == pytest.approx(0.5 * np.mean((p - t) ** 2))
    e = _rand(rng, 5, 6)
    assert np.sum(g * e) == pytest.approx(cnn.mse(p + 1e-30j * e, t)[0].imag / 1e-30, rel=1e-12)


def test_adam_step_by_hand():
    # first step: m = 0.1 g, v = 0.001 g^2, bias-corrected to g and g^2: update = lr * g / (|g| + eps)
    th, m, v = cnn.adam_step(np.array([1.0]), np.array([0.5]), np.zeros(1), np.zeros(1), 1, lr=0.1)
    assert th[0] == pytest.approx(1.0 - 0.1 * 0.5 / (0.5 + 1e-8), rel=1e-14)
    assert m[0] == pytest.approx(0.05) and v[0] == pytest.approx(0.00025)
    # second step with g = -0.5
    th2, m2, v2 = cnn.adam_step(th, np.array([-0.5]), m, v, 2, lr=0.1)
    mh = (0.9 * 0.05 - 0.05) / (1 - 0.81)
    vh = (0.999 * 0.00025 + 0.001 * 0.25) / (1 - 0.998001)
    assert th2[0] == pytest.approx(th[0] - 0.1 * mh / (np.sqrt(vh) + 1e-8), rel=1e-13)


def test_bf16_round_matches_torch_conversion():
    import torch

    rng = np.random.default_rng(11)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-20, 20, 10000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).float().double().numpy()
    np.testing.assert_array_equal(cnn.bf16_round(x), want)
