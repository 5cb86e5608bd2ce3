"""FP64 CPU oracle for the template surrogate network.

TEST INFRASTRUCTURE ONLY: used by the tests (gradient and step checks of the CUDA
training kernels) and never by the product path.

Network: x (6) -> [Linear 256, GELU] x 4 -> Linear 320.  GELU(z) = z (1 + erf(z / sqrt 2)) / 2.
Quantisation points (part of the surrogate's definition): every operand of every matrix
product is rounded to BF16 (round to nearest even): weights and layer inputs in the forward
pass, the back-propagated gradients and the weights in the backward pass; products are
summed exactly here (FP32 on the GPU); bias gradients sum the unrounded gradients.  Loss: mean squared error over the batch and the 320 outputs.
Optimiser: Adam with bias correction on FP32 master weights (Kingma & Ba 2015).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SIZES = (6, 256, 256, 256, 256, 320)


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    nan = np.isnan(f)
    out = np.where(nan, f, out)
    return out.astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def init_params(seed: int = 0):
    """Weights W_l [out, in] ~ U(-1/sqrt(in), 1/sqrt(in)) from a seeded generator, biases 0."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 77]))
    ws, bs = [], []
    for fi, fo in zip(SIZES[:-1], SIZES[1:]):
        lim = 1.0 / math.sqrt(fi)
        ws.append(rng.uniform(-lim, lim, (fo, fi)).astype(np.float32).astype(np.float64))
        bs.append(np.zeros(fo))
    return ws, bs


def forward(ws, bs, x, quantize: bool = True):
    """Pre-activations z_l and layer inputs a_l (BF16-rounded) for every layer; returns (out, cache).
    quantize=False skips the BF16 rounding (used to check the chain rule by finite differences)."""
    q = bf16 if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    a = q(x)
    cache = []
    n_layers = len(ws)
    for li, (w, b) in enumerate(zip(ws, bs)):
        z = a @ q(w).T + b
        cache.append((a, z))
        if li < n_layers - 1:
            a = q(gelu(z))
        else:
            a = z
    return a, cache


def loss_and_grads(ws, bs, x, y, quantize: bool = True):
    """MSE loss and its gradients with respect to the FP32 master weights and biases; the BF16
    rounding points pass gradients straight through."""
    q = bf16 if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    out, cache = forward(ws, bs, x, quantize)
    m = x.shape[0]
    diff = out - y
    loss = float(np.mean(diff * diff))
    g = 2.0 * diff / diff.size                     # dL/d out
    gws, gbs = [None] * len(ws), [None] * len(ws)
    for li in range(len(ws) - 1, -1, -1):
        a, z = cache[li]
        if li < len(ws) - 1:
            g = g * gelu_grad(z)
        gq = q(g)
        gws[li] = gq.T @ a
        gbs[li] = g.sum(axis=0)
        if li > 0:
            g = gq @ q(ws[li])
    return loss, gws, gbs


def adam_step(ws, bs, gws, gbs, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of every weight and bias (state: dict with t, m, v lists)."""
    state["t"] += 1
    t = state["t"]
    params = ws + bs
    grads = gws + gbs
    for i, (p, g) in enumerate(zip(params, grads)):
        state["m"][i] = b1 * state["m"][i] + (1 - b1) * g
        state["v"][i] = b2 * state["v"][i] + (1 - b2) * g * g
        mh = state["m"][i] / (1 - b1 ** t)
        vh = state["v"][i] / (1 - b2 ** t)
        p -= lr * mh / (np.sqrt(vh) + eps)
    return ws, bs


def adam_state(ws, bs):
    return {"t": 0, "m": [np.zeros_like(p) for p in ws + bs], "v": [np.zeros_like(p) for p in ws + bs]}
