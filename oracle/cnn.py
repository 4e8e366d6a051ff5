"""The learned right preconditioner: a 6-layer 3x3 convolutional network in FP64 numpy.

Not in the paper (an addition on top of its GMRES use).  Layers 1..6 map channels
1 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1 with 3x3 kernels, zero padding and no bias; a ReLU
follows layers 1..5.  With no bias the network is positively homogeneous, so the
preconditioner M(r) = rms(r) * net(r / rms(r)) equals net(r) in exact arithmetic; the
scaling only keeps reduced-precision activations in range.

Training loss for a batch of (residual r_b, correction e_b) pairs:
    L = (1/B) sum_b ||net(r_b) - e_b||^2 / ||e_b||^2.

Pins: tests/test_oracle_cnn.py (central finite differences of L for weight and input
gradients; a 1x1-equivalent kernel against a hand-computed stencil; homogeneity).
"""
from __future__ import annotations

import numpy as np

CHANNELS = (1, 32, 32, 32, 32, 32, 1)


def init_weights(seed: int = 0, channels=CHANNELS):
    """He-normal 3x3 weights, shape (C_out, C_in, 3, 3) per layer, float64."""
    rng = np.random.default_rng(seed)
    ws = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        std = np.sqrt(2.0 / (cin * 9))
        ws.append(rng.standard_normal((cout, cin, 3, 3)) * std)
    return ws


def conv3x3(x, W):
    """Zero-padded 3x3 cross-correlation: x (B, Cin, H, W) -> (B, Cout, H, W)."""
    B, C, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    out = np.zeros((B, W.shape[0], H, Wd))
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("oc,bchw->bohw", W[:, :, dy, dx], xp[:, :, dy:dy + H, dx:dx + Wd])
    return out


def conv3x3_backward(x, W, gout):
    """Gradients of sum(gout * conv3x3(x, W)) with respect to W and x."""
    B, C, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    gW = np.zeros_like(W)
    gxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            gW[:, :, dy, dx] = np.einsum("bohw,bchw->oc", gout, xp[:, :, dy:dy + H, dx:dx + Wd])
            gxp[:, :, dy:dy + H, dx:dx + Wd] += np.einsum("oc,bohw->bchw", W[:, :, dy, dx], gout)
    return gW, gxp[:, :, 1:-1, 1:-1]


def forward(ws, x):
    """Network output and the per-layer inputs (kept for the backward pass)."""
    acts = [x]
    h = x
    for li, W in enumerate(ws):
        h = conv3x3(h, W)
        if li < len(ws) - 1:
            h = np.maximum(h, 0.0)
        acts.append(h)
    return h, acts


def loss_and_grads(ws, r, e):
    """Loss L and dL/dW per layer, dL/dr.  r, e: (B, 1, H, W)."""
    B = r.shape[0]
    y, acts = forward(ws, r)
    diff = y - e
    en = np.sum(e * e, axis=(1, 2, 3))
    L = float(np.mean(np.sum(diff * diff, axis=(1, 2, 3)) / en))
    g = (2.0 / B) * diff / en[:, None, None, None]
    grads = [None] * len(ws)
    for li in range(len(ws) - 1, -1, -1):
        if li < len(ws) - 1:
            g = g * (acts[li + 1] > 0.0)
        gW, g = conv3x3_backward(acts[li], ws[li], g)
        grads[li] = gW
    return L, grads, g


def apply_preconditioner(ws, r_vec, H, W):
    """M(r) for one residual vector (length H*W, row-major grid), with RMS scaling."""
    x = np.asarray(r_vec, dtype=np.float64).reshape(1, 1, H, W)
    s = np.sqrt(np.mean(x * x))
    if s == 0.0:
        return np.zeros(H * W)
    y, _ = forward(ws, x / s)
    return (y * s).reshape(H * W)


def _round_bf16(x):
    """Round float64 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16_storage(ws, x):
    """The network with BF16 weights and BF16-stored hidden activations (what the GPU
    kernels keep in memory): weights rounded to bfloat16, each hidden layer's ReLU output
    rounded to bfloat16, sums in FP64; input and output stay unrounded."""
    wb = [_round_bf16(W) for W in ws]
    h = x
    acts = [x]
    for li, W in enumerate(wb):
        h = conv3x3(h, W)
        if li < len(wb) - 1:
            h = _round_bf16(np.maximum(h, 0.0))
        acts.append(h)
    return h, acts


def loss_and_grads_bf16_storage(ws, r, e):
    """loss_and_grads with the GPU's storage rounding: BF16 weights, BF16 hidden
    activations and BF16 hidden-layer gradients dL/dz (the output gradient stays FP64)."""
    B = r.shape[0]
    wb = [_round_bf16(W) for W in ws]
    y, acts = forward_bf16_storage(ws, r)
    diff = y - e
    en = np.sum(e * e, axis=(1, 2, 3))
    L = float(np.mean(np.sum(diff * diff, axis=(1, 2, 3)) / en))
    g = (2.0 / B) * diff / en[:, None, None, None]
    grads = [None] * len(ws)
    for li in range(len(ws) - 1, -1, -1):
        if li < len(ws) - 1:
            g = _round_bf16(g * (acts[li + 1] > 0.0))
        gW, g = conv3x3_backward(acts[li], wb[li], g)
        grads[li] = gW
    return L, grads, y
