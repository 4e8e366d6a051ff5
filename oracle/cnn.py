"""The learned right preconditioner: a 6-layer 3x3 convolutional network in FP64 numpy.

Not in the paper (an addition on top of its GMRES use).  Layers 1..6 map channels
1 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1 with 3x3 kernels, zero padding and no bias; a ReLU
follows layers 1..5.  With no bias the network is positively homogeneous:
s net(x / s) = net(x) for s > 0 in exact arithmetic, so scaling its input by the RMS
only keeps reduced-precision activations in range.

Two training losses for a batch of (residual r_b, correction e_b) pairs, A e_b = r_b:
    regression:  L = (1/B) sum_b ||net(r_b) - e_b||^2 / ||e_b||^2;
    residual:    L = (1/B) sum_b ||A (x_b + net(x_b)) - r_b||^2 / ||r_b||^2, with
                 x_b = D^{-1} r_b the Jacobi-scaled residual: the error of the correction
                 M(r_b) - e_b measured in the norm ||A .||, which needs no e_b.
The preconditioner that the residual loss trains (fgmres):
    M(w) = u + s net(u / s),   u = D^{-1} w,  s = rms(u),
the Jacobi step plus the learned correction (D = diag(A)).

Pins: tests/test_oracle_cnn.py (central finite differences of both losses for weight and
input gradients; a 1x1-equivalent kernel against a hand-computed stencil; homogeneity;
a network that computes c x exactly, giving closed-form losses and M(w) = (1 + c) D^{-1} w;
zero weights giving the Jacobi preconditioner).  The BF16-storage variants
(forward_bf16_storage, loss_and_grads_bf16_storage, backward(bf16=True), the residual loss
with bf16=True): a 1 x 1-image chain of three layers whose output, loss and gradients are
written in closed form on rationals with every rounding point changing its value, and
dyadic weights and inputs for which nothing rounds, where they equal the FP64 functions
bit for bit; the rounding itself is gmres.round_bf16 (golden values).

This module is test infrastructure: only tests, the smoke check and the CPU baseline of
the benchmark use it.
"""
from __future__ import annotations

import numpy as np

from .gmres import round_bf16

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


def _round_bf16(x):
    """Round to the nearest bfloat16 (ties to even), as float64: the value is first taken to
    float32 (the GPU's accumulator type) and then rounded by gmres.round_bf16, whose
    results are pinned by golden values."""
    return round_bf16(np.asarray(x, dtype=np.float64).astype(np.float32)).astype(np.float64)


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
    activations and BF16 hidden-layer gradients dL/dz (the output gradient stays FP64).
    Returns L, dL/dW per layer and the network output y."""
    B = r.shape[0]
    y, acts = forward_bf16_storage(ws, r)
    diff = y - e
    en = np.sum(e * e, axis=(1, 2, 3))
    L = float(np.mean(np.sum(diff * diff, axis=(1, 2, 3)) / en))
    g = (2.0 / B) * diff / en[:, None, None, None]
    grads, _ = backward(ws, acts, g, bf16=True)
    return L, grads, y


def backward(ws, acts, gy, bf16=False):
    """dL/dW per layer and dL/dx from dL/dy, after forward (or forward_bf16_storage when
    `bf16`: BF16 weights and BF16-rounded hidden-layer gradients, as on the GPU)."""
    wl = [_round_bf16(W) for W in ws] if bf16 else ws
    g = gy
    grads = [None] * len(ws)
    for li in range(len(ws) - 1, -1, -1):
        if li < len(ws) - 1:
            g = g * (acts[li + 1] > 0.0)
            if bf16:
                g = _round_bf16(g)
        gW, g = conv3x3_backward(acts[li], wl[li], g)
        grads[li] = gW
    return grads, g


def residual_loss_and_grads(ws, x, r, A, bf16=False):
    """Residual loss of a batch (see the module docstring): x, r (B, 1, H, W) with x the
    network input and r the residual it should remove; A a sparse or dense (H W x H W)
    operator shared by the batch.  Returns L, dL/dW per layer, dL/dx (through z = x + y)
    and the network output y."""
    B = x.shape[0]
    y, acts = forward_bf16_storage(ws, x) if bf16 else forward(ws, x)
    z = (x + y).reshape(B, -1)
    rr = r.reshape(B, -1)
    res = np.stack([A @ z[b] for b in range(B)]) - rr
    rn = np.sum(rr * rr, axis=1)
    L = float(np.mean(np.sum(res * res, axis=1) / rn))
    AT = A.T
    gy = np.stack([AT @ res[b] for b in range(B)]) * (2.0 / B) / rn[:, None]
    gy = gy.reshape(y.shape)
    grads, gx = backward(ws, acts, gy, bf16=bf16)
    return L, grads, gx + gy, y


def jacobi_network_preconditioner(ws, w, dinv, H, W, bf16=False):
    """M(w) = u + s net(u / s) with u = D^{-1} w (dinv: the inverse diagonal) and
    s = rms(u); the Jacobi step alone when the network output is zero."""
    u = np.asarray(w, dtype=np.float64) * dinv
    s = np.sqrt(np.mean(u * u))
    if s == 0.0:
        return u
    x = (u / s).reshape(1, 1, H, W)
    y, _ = forward_bf16_storage(ws, x) if bf16 else forward(ws, x)
    return u + y.reshape(H * W) * s


def inverse_diagonal(A):
    """1 / a_ii for every row of a scipy sparse matrix (1 where the diagonal is 0)."""
    d = np.asarray(A.diagonal(), dtype=np.float64)
    out = np.ones_like(d)
    nz = d != 0.0
    out[nz] = 1.0 / d[nz]
    return out
