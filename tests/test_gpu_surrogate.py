"""The surrogate network's CUDA kernels against the FP64 oracle (same BF16 rounding points).

Tolerances: both sides round the same operands to BF16; the GPU accumulates in FP32 and may
round an activation or gradient to the neighbouring BF16 value where the FP32 and FP64 sums
straddle a rounding boundary (relative 2^-8 on that element).  Norm-wise relative errors of
a few 1e-3 cover that; index or transpose mistakes give O(1) errors.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2202_11839_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def _setup(batch=64, seed=5):
    import torch
    from paper_2202_11839_gb300 import lpp as L
    L.load_library()
    layers = S.surrogate_init(seed)
    rng = np.random.default_rng(seed)
    layers = [(w, (rng.standard_normal(b.shape) * 0.05).astype(np.float32)) for w, b in layers]
    x = rng.uniform(-1, 1, (batch, 6)).astype(np.float32)
    y = rng.standard_normal((batch, 320)).astype(np.float32)
    net = L.Surrogate(L.flatten_params(layers), batch=batch)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return L, net, layers, x, y, t


def _oracle_params(layers):
    return [w.astype(np.float64) for w, b in layers], [b.astype(np.float64) for w, b in layers]


def test_forward_matches_oracle():
    L, net, layers, x, y, t = _setup()
    out = net.infer(t(x)).cpu().numpy()
    ws, bs = _oracle_params(layers)
    ref, _ = M.forward(ws, bs, x.astype(np.float64))
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 2e-3
    net.close()


def test_gradients_match_oracle():
    import torch
    L, net, layers, x, y, t = _setup()
    idx = t(np.arange(64, dtype=np.int32))
    g, loss = net.gradients(t(x), t(y), idx)
    ws, bs = _oracle_params(layers)
    rl, gws, gbs = M.loss_and_grads(ws, bs, x.astype(np.float64), y.astype(np.float64))
    assert abs(loss - rl) <= 1e-4 * rl
    got = L.unflatten_params(g)
    for li in range(5):
        gw, gb = got[li]
        ew = np.linalg.norm(gw - gws[li]) / np.linalg.norm(gws[li])
        eb = np.linalg.norm(gb - gbs[li]) / np.linalg.norm(gbs[li])
        assert ew < 5e-3 and eb < 5e-3, (li, ew, eb)
    # the network is unchanged by the gradient call
    np.testing.assert_array_equal(net.params(), L.flatten_params(layers))
    net.close()


def test_one_adam_step_matches_oracle():
    import torch
    L, net, layers, x, y, t = _setup()
    sched = t(np.arange(64, dtype=np.int32))
    losses = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.train(t(x), t(y), sched, 1e-3, losses)
    torch.cuda.synchronize()
    ws, bs = _oracle_params(layers)
    rl, gws, gbs = M.loss_and_grads(ws, bs, x.astype(np.float64), y.astype(np.float64))
    st = M.adam_state(ws, bs)
    M.adam_step(ws, bs, gws, gbs, st, lr=1e-3)
    got = L.unflatten_params(net.params())
    for li in range(5):
        w0, b0 = layers[li]
        dw_gpu = got[li][0] - w0
        dw_ref = ws[li] - w0
        # Adam's first step is +-lr per element wherever the gradient is not tiny; compare the moves
        agree = np.mean(np.sign(dw_gpu) == np.sign(dw_ref))
        assert agree > 0.99, (li, agree)
        assert np.max(np.abs(dw_gpu - dw_ref)) < 1.5e-3
    assert abs(float(losses[0]) - rl) <= 1e-4 * rl
    net.close()


def test_training_reduces_the_loss():
    import torch
    from paper_2202_11839_gb300 import lpp as L
    L.load_library()
    rng = np.random.default_rng(8)
    n = 2048
    x = rng.uniform(-1, 1, (n, 6)).astype(np.float32)
    basis = rng.standard_normal((6, 320)).astype(np.float32) / 3
    y = np.tanh(x @ basis).astype(np.float32)
    net = L.Surrogate(L.flatten_params(S.surrogate_init(1)), batch=128)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    steps = 400
    sched = np.concatenate([rng.permutation(n)[:128] for _ in range(steps)]).astype(np.int32)
    losses = torch.zeros(steps, dtype=torch.float64, device="cuda")
    net.train(t(x), t(y), t(sched), 2e-3, losses)
    l = losses.cpu().numpy()
    assert l[-20:].mean() < 0.05 * l[:5].mean(), (l[:5], l[-20:])
    net.close()
