"""Pins for the surrogate-network oracle: BF16 rounding, GELU derivative and gradients."""
import math

import numpy as np
import torch

from oracle import mlp_oracle as M


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(10000) * 10 ** rng.uniform(-6, 6, 10000)
    x = np.concatenate([x, [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 3.0e38]])
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.bf16(x), want)


def test_gelu_grad_by_finite_differences():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(M.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)


def test_gradients_by_finite_differences():
    """Without the BF16 points the network is smooth: every gradient (weights and biases of
    all five layers) matches central differences of the loss."""
    rng = np.random.default_rng(1)
    ws, bs = M.init_params(3)
    bs = [rng.standard_normal(b.shape) * 0.1 for b in bs]
    x = rng.uniform(-1, 1, (5, 6))
    y = rng.standard_normal((5, 320))
    loss, gws, gbs = M.loss_and_grads(ws, bs, x, y, quantize=False)
    h = 1e-5
    for li in range(5):
        for (i, j) in ((0, 0), (3, 1), (ws[li].shape[0] - 1, ws[li].shape[1] - 1)):
            wp = [w.copy() for w in ws]
            wm = [w.copy() for w in ws]
            wp[li][i, j] += h
            wm[li][i, j] -= h
            fd = (M.loss_and_grads(wp, bs, x, y, False)[0] - M.loss_and_grads(wm, bs, x, y, False)[0]) / (2 * h)
            assert abs(gws[li][i, j] - fd) <= 1e-6 * abs(fd) + 1e-10, (li, i, j, gws[li][i, j], fd)
        j = 2
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[li][j] += h
        bm[li][j] -= h
        fd = (M.loss_and_grads(ws, bp, x, y, False)[0] - M.loss_and_grads(ws, bm, x, y, False)[0]) / (2 * h)
        assert abs(gbs[li][j] - fd) <= 1e-6 * abs(fd) + 1e-10, (li, gbs[li][j], fd)


def test_adam_first_step_is_signed_lr():
    """With bias correction the first Adam step moves every parameter by lr * sign(grad)."""
    ws, bs = M.init_params(0)
    rng = np.random.default_rng(2)
    gws = [rng.standard_normal(w.shape) for w in ws]
    gbs = [rng.standard_normal(b.shape) for b in bs]
    w0 = [w.copy() for w in ws]
    st = M.adam_state(ws, bs)
    M.adam_step(ws, bs, gws, gbs, st, lr=1e-3)
    for w, w_old, g in zip(ws, w0, gws):
        np.testing.assert_allclose(w - w_old, -1e-3 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-9)
