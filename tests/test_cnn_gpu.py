"""Parity of the start-model network's layers (libfwi CNN kernels, tcgen05
tensor-core GEMMs through the C ABI) with the FP64 reference layers of
oracle/cnn.py, and of the GEMM itself with an FP64 product of the same
BF16-rounded operands.

The GEMMs multiply BF16-rounded operands with FP32 accumulation, so the oracle
is evaluated on the same BF16-rounded operands (oracle.cnn.bf16_round) and the
remaining difference is FP32 accumulation: relative L2 <= 1e-5. Upsampling is
exact; MSE and Adam are FP32 element-wise against FP64 (1e-6)."""

import numpy as np
import pytest

from oracle import cnn

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _cuda(a):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


GEMMS = [  # M, N, K, splits, bias+relu, row padding of A and B
    (128, 16, 64, 1, False, 0),
    (300, 40, 200, 1, True, 8),
    (1000, 256, 1152, 1, True, 0),
    (77, 300, 16, 1, False, 16),
    (144, 32, 5000, 8, False, 0),
    (27, 5, 442, 3, False, 24),
    (1, 1, 1, 1, True, 0),       # degenerate: one row, one column, one term (all zero-filled to the tile)
    (129, 17, 8, 1, False, 0),   # one row past a tile; N one past a multiple of 16
    (5, 256, 70, 2, False, 0),   # N at the single-tile maximum; split K with a ragged last block
]


@pytest.mark.parametrize("case", GEMMS, ids=[f"{c[0]}x{c[1]}x{c[2]}-s{c[3]}" for c in GEMMS])
def test_tcgen05_gemm(fwi_lib, case):
    """out[n][m] = act(sum_k A[m][k] B[n][k] + bias[n]) on BF16 operands with
    FP32 accumulation: ragged M, N, K (zero fill at the tile edges), N over
    several tiles, split K, strided operands."""
    import torch

    from paper_2003_06027_gb300 import learned as L

    M, N, K, splits, act, pad = case
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    a = rng.standard_normal((M, K)).astype(np.float32)
    b = rng.standard_normal((N, K)).astype(np.float32)
    bias = rng.standard_normal(N).astype(np.float32)
    lda = (K + 7) // 8 * 8 + pad
    h = L.Handle(0)
    Ab = torch.zeros((M, lda), dtype=torch.int16, device="cuda")
    Bb = torch.zeros((N, lda), dtype=torch.int16, device="cuda")
    Ab[:, :K] = L.to_bf16(_cuda(a))
    Bb[:, :K] = L.to_bf16(_cuda(b))
    out = L.gemm_bt(h, Ab[:, :K], Bb[:, :K], bias=_cuda(bias) if act else None, relu=act, splits=splits)
    h.check()
    want = np.float64(cnn.bf16_round(b)) @ np.float64(cnn.bf16_round(a)).T
    if act:
        want = np.maximum(want + np.float64(bias)[:, None], 0.0)
    got = out.cpu().numpy()
    assert got.shape == (N, M)
    assert np.isfinite(got).all()
    assert rel(got, want) <= 1e-5
    again = L.gemm_bt(h, Ab[:, :K], Bb[:, :K], bias=_cuda(bias) if act else None, relu=act, splits=splits)
    assert torch.equal(again, out)  # deterministic: fixed-order split sums, no atomics


SHAPES = [  # C, B, H, W, O, sh, sw, relu
    (3, 2, 17, 13, 5, 1, 1, True),
    (16, 3, 40, 16, 8, 4, 1, True),
    (8, 2, 25, 12, 16, 2, 2, False),
    (32, 1, 9, 33, 4, 2, 1, True),
    (64, 2, 16, 32, 32, 1, 1, True),
    (20, 3, 7, 40, 24, 1, 1, False),
    (8, 3, 20, 64, 4, 2, 2, True),  # stride 2, 8-pixel tap-major runs over two staged row blocks
    # rows wider than the row-staged im2col's shared memory, and a column stride of 8:
    # the per-element im2col kernels
    (2, 1, 5, 4100, 3, 1, 1, True),
    (3, 1, 9, 70, 4, 1, 8, False),
]


@pytest.mark.parametrize("shape", SHAPES, ids=[f"{s[0]}x{s[1]}x{s[2]}x{s[3]}-o{s[4]}-s{s[5]}{s[6]}" for s in SHAPES])
def test_conv_forward_backward(fwi_lib, shape):
    from paper_2003_06027_gb300 import learned as L

    C, B, H, W, O, sh, sw, relu = shape
    rng = np.random.default_rng(C * 100 + H)
    x = rng.standard_normal((C, B, H, W)).astype(np.float32)
    w = (rng.standard_normal((O, C, 3, 3)) * 0.3).astype(np.float32)
    b = rng.standard_normal(O).astype(np.float32) * 0.1
    h = L.Handle(0)
    wb = L.to_bf16(_cuda(w))
    y = L.conv_forward(h, _cuda(x), wb, _cuda(b), sh, sw, relu)
    xr, wr = cnn.bf16_round(x), cnn.bf16_round(w)
    pre = cnn.conv2d(xr, wr, np.float64(b), sh, sw)
    want = cnn.relu(pre) if relu else pre
    assert y.shape == want.shape
    assert rel(y.cpu().numpy(), want) <= 1e-5

    dy = rng.standard_normal(want.shape).astype(np.float32)
    dyt = _cuda(dy)
    dx, dw, db = L.conv_backward(h, _cuda(x), wb, y, dyt, sh, sw, relu, need_dx=True)
    g = cnn.relu_backward(y.cpu().numpy().astype(np.float64), dy) if relu else np.float64(dy)
    # dy is overwritten with the pre-activation gradient (FP32, before rounding)
    np.testing.assert_array_equal(dyt.cpu().numpy(), np.float32(g))
    dxo, dwo, dbo = cnn.conv2d_backward(xr, wr, cnn.bf16_round(np.float32(g)), sh, sw)
    assert rel(dx.cpu().numpy(), dxo) <= 1e-5
    assert rel(dw.cpu().numpy(), dwo) <= 1e-5
    assert rel(db.cpu().numpy(), g.sum(axis=(1, 2, 3))) <= 1e-6
    _, dw2, _ = L.conv_backward(h, _cuda(x), wb, y, _cuda(dy), sh, sw, relu, need_dx=False)
    h.check()
    assert np.array_equal(dw2.cpu().numpy(), dw.cpu().numpy())


GATHER_SHAPES = SHAPES[:-2] + [  # the gathered operand also for a full 64-channel layer of the network's size class
    (64, 2, 64, 128, 32, 1, 1, True),
    (1, 3, 37, 29, 16, 2, 1, True),
]


@pytest.mark.parametrize("shape", GATHER_SHAPES, ids=[f"{s[0]}x{s[1]}x{s[2]}x{s[3]}-o{s[4]}-s{s[5]}{s[6]}"
                                                       for s in GATHER_SHAPES])
def test_gathered_operand_equals_im2col(fwi_lib, shape):
    """The convolution GEMMs with their tap operand gathered from the
    activations inside the GEMM (the default) give the forward output and the
    stride-1 data gradient of the im2col-matrix path bit for bit: the same
    BF16 operand, the same MMA order; every tile row, edge and padding tap."""
    import torch

    from paper_2003_06027_gb300 import learned as L

    C, B, H, W, O, sh, sw, relu = shape
    rng = np.random.default_rng(C * 31 + W)
    x = _cuda(rng.standard_normal((C, B, H, W)).astype(np.float32))
    wb = L.to_bf16(_cuda((rng.standard_normal((O, C, 3, 3)) * 0.3).astype(np.float32)))
    b = _cuda(rng.standard_normal(O).astype(np.float32) * 0.1)
    out = {}
    for gather in (True, False):
        h = L.Handle(0)
        h.set_conv_gather(gather)
        y = L.conv_forward(h, x, wb, b, sh, sw, relu)
        dy = _cuda(np.random.default_rng(7).standard_normal(tuple(y.shape)).astype(np.float32))
        dx, dw, db = L.conv_backward(h, x, wb, y, dy, sh, sw, relu, need_dx=True)
        h.check()
        out[gather] = (y, dx, dw, db)
    for a, c in zip(out[True], out[False]):
        assert torch.equal(a, c)
    assert torch.isfinite(out[True][0]).all()


def test_upsample_and_mse_and_adam(fwi_lib):
    from paper_2003_06027_gb300 import learned as L

    rng = np.random.default_rng(9)
    x = rng.standard_normal((3, 2, 5, 7)).astype(np.float32)
    u = L.upsample2(_cuda(x)).cpu().numpy()
    np.testing.assert_array_equal(u, cnn.upsample2(x))
    d = rng.standard_normal(u.shape).astype(np.float32)
    np.testing.assert_allclose(L.upsample2_backward(_cuda(d)).cpu().numpy(), cnn.upsample2_backward(np.float64(d)),
                               rtol=1e-6, atol=1e-6)
    xw = rng.standard_normal((4, 2, 40, 300)).astype(np.float32)  # rows wider than a block of threads
    np.testing.assert_array_equal(L.upsample2(_cuda(xw)).cpu().numpy(), cnn.upsample2(xw))
    dw_ = rng.standard_normal((4, 2, 80, 600)).astype(np.float32)
    np.testing.assert_allclose(L.upsample2_backward(_cuda(dw_)).cpu().numpy(),
                               cnn.upsample2_backward(np.float64(dw_)), rtol=1e-6, atol=1e-6)
    h = L.Handle(0)
    for n in (5000, 1_000_003):  # one block's worth, and many blocks with a ragged tail
        p, t = rng.standard_normal(n).astype(np.float32), rng.standard_normal(n).astype(np.float32)
        loss, dp = L.mse(h, _cuda(p), _cuda(t))
        lo, go = cnn.mse(np.float64(p), np.float64(t))
        assert float(loss[0]) == pytest.approx(lo, rel=1e-6)  # FP32 residuals, FP64 sum
        assert rel(dp.cpu().numpy(), go) <= 1e-6
    th, g = rng.standard_normal(777).astype(np.float32), rng.standard_normal(777).astype(np.float32)
    tt, gg, m, v = _cuda(th), _cuda(g), _cuda(np.zeros(777)), _cuda(np.zeros(777))
    thb = L.to_bf16(tt)
    want, mo, vo = np.float64(th), np.zeros(777), np.zeros(777)
    for step in (1, 2, 3):
        L._chk(L._lib().fwi_cnn_adam(L._p(tt), L._p(gg), L._p(m), L._p(v), 777, step, 1e-2, 0.9, 0.999, 1e-8,
                                     L._p(thb), L._st()))
        want, mo, vo = cnn.adam_step(want, np.float64(g), mo, vo, step, 1e-2)
    assert rel(tt.cpu().numpy(), want) <= 1e-6
    assert np.array_equal(thb.cpu().numpy().view(np.uint16),
                          (cnn.bf16_round(tt.cpu().numpy()).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16))


def test_network_learns_layered_models(fwi_lib):
    """A short training run on solver-generated gathers lowers the loss, and the
    network beats the best constant model on held-out surveys."""
    import torch

    from paper_2003_06027_gb300 import learned as L

    X, Y, _ = L.make_dataset(192, seed=101)
    Xt, Yt, _ = L.make_dataset(16, seed=202)
    net = L.Net(0, seed=1)
    log = L.train(net, X, Y, epochs=6, batch=16, lr=1e-3)
    assert np.isfinite(log.loss).all()
    assert np.mean(log.loss[-5:]) < 0.5 * np.mean(log.loss[:5])
    with torch.no_grad():
        pred = net.forward(Xt)
        err_net = float(((pred - Yt) ** 2).mean())
        err_const = float(((Yt.mean() - Yt) ** 2).mean())
    assert err_net < err_const, (err_net, err_const)


def test_learned_start_gains_over_the_start_without_it(fwi_lib):
    """What the trained network gains: on held-out surveys, FWI (L-BFGS, same
    iteration budget) from the network's prediction against FWI from the start
    available without the network (the mean of the training models, which uses
    no survey information). The learned start must be closer to the true model
    and end at a clearly lower misfit. The comparison with the smoothed true
    model (which is built from the answer) is reported, not asserted."""
    from paper_2003_06027_gb300 import learned as L

    X, Y, _ = L.make_dataset(3072, seed=303)
    net = L.Net(0, seed=3)
    L.train(net, X, Y, epochs=12, batch=32, lr=1e-3)
    mean_model = (L.V_MID + L.V_HALF * Y[0].mean(dim=0)).contiguous()
    del X, Y
    _, s = L.compare_fwi(net, n_models=3, seed=404, iters=12, mean_model=mean_model)
    print("\nlearned start vs mean-model start:", {k: s[k] for k in (
        "learned_start_model_error", "mean_start_model_error", "learned_final_misfit", "mean_final_misfit",
        "plain_final_misfit", "learned_seconds_to_plain_final", "plain_fwi_seconds")})
    assert s["learned_start_model_error"] < s["mean_start_model_error"]
    assert s["learned_final_misfit"] < 0.5 * s["mean_final_misfit"]
