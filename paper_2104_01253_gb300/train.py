"""Training the convolutional preconditioner on the GPU (orchestration of C-ABI calls).

Data: for each seeded operator of the variable-coefficient family (synth.varcoef_fields_2d),
plain DCGS2-GMRES(n) (gmres_solve), one restart cycle per call, records the residual
r_j = b - A x_j at every restart.  Each r_j is a (residual, correction) pair with the
correction e_j = A^{-1} r_j left implicit: the residual loss

    L = (1/B) sum_b ||A (x_b + net(x_b)) - r_b||^2 / ||r_b||^2,   x_b = D^{-1} r_b,

is ||A (M(r_b) - e_b)||^2 / ||r_b||^2 for the preconditioner M that fgmres_solve applies
(M(w) = D^{-1} w + s net(D^{-1} w / s)), so it needs r_b and A only.  Inputs and residuals
of a sample are divided by s = rms(D^{-1} r_b) (the network is positively homogeneous).
The residual, its Jacobi scaling and s come from libkrylov (kc_cnn_residual_sample), and
every forward, backward and Adam update runs there too (kc_cnn_train_step_residual);
each step draws its batch from one operator, cycling through the training operators.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (Context, DeviceCSR, gmres_solve, kc_cnn_param_count, kc_cnn_residual_sample,
               kc_cnn_train_step_residual)


def varcoef_operator(N: int, seed: int):
    from synth import convdiff_csr, varcoef_fields_2d
    kappa, wind = varcoef_fields_2d(N, seed)
    return convdiff_csr(N, 2, wind, kappa=kappa)


def he_init(seed: int) -> np.ndarray:
    """He-normal weights in the library's packed layout ([Cout][3][3][Cin] per layer)."""
    rng = np.random.default_rng(seed)
    chans = (1, 32, 32, 32, 32, 32, 1)
    parts = []
    for cin, cout in zip(chans[:-1], chans[1:]):
        parts.append(rng.standard_normal(cout * 9 * cin) * np.sqrt(2.0 / (9 * cin)))
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == kc_cnn_param_count()
    return w


def generate_pairs(ctx: Context, N: int, seeds, restart: int = 40, max_cycles: int = 20,
                   rhs_seed_offset: int = 1000, host_ops=None, on_device: bool = False):
    """Restart residuals of plain GMRES solves on the seeded operators (host_ops: the host
    CSR operators of `seeds`, if already built).

    Returns (ops, X, R, owner): the device operators, the network inputs
    X = D^{-1} r / s and residuals R = r / s (float32, (n, 1, N, N); host arrays, or device
    tensors with on_device), and the index of each sample's operator.  A sample's cycle
    within its operator's solve is its rank among the samples of that operator."""
    from synth import gaussian_vector
    ops, X, R, owner = [], [], [], []
    seeds = list(seeds)
    if on_device:                                    # capacity: every cycle of every solve
        Xd = torch.empty((len(seeds) * max_cycles, N * N), dtype=torch.float32, device="cuda")
        Rd = torch.empty_like(Xd)
    for oi, seed in enumerate(seeds):
        Ah = host_ops[oi] if host_ops is not None else varcoef_operator(N, seed)
        A = DeviceCSR(Ah)
        ops.append(A)
        b = torch.as_tensor(gaussian_vector(Ah.m, rhs_seed_offset + seed), device="cuda")
        x = torch.zeros_like(b)
        xin = torch.empty(Ah.m, dtype=torch.float32, device="cuda")
        res = torch.empty_like(xin)
        bnorm = None
        for _ in range(max_cycles):
            rn = kc_cnn_residual_sample(ctx, A, b, x, xin, res)
            bnorm = rn if bnorm is None else bnorm           # x = 0 on the first pass
            if rn <= 1e-9 * bnorm:
                break
            if on_device:
                Xd[len(owner)].copy_(xin)
                Rd[len(owner)].copy_(res)
            else:
                X.append(xin.cpu().numpy())
                R.append(res.cpu().numpy())
            owner.append(oi)
            gmres_solve(ctx, A, b, x, restart=restart, rtol=1e-10, maxit=restart)
    if on_device:
        n = len(owner)
        return ops, Xd[:n].view(n, 1, N, N), Rd[:n].view(n, 1, N, N), np.asarray(owner)
    X = np.stack(X).reshape(-1, 1, N, N)
    R = np.stack(R).reshape(-1, 1, N, N)
    return ops, X, R, np.asarray(owner)


def train(ctx: Context, ops, X, R, owner: np.ndarray, steps: int = 600, batch: int = 16,
          lr: float = 2e-3, seed: int = 0, w0=None, select=None):
    """Adam on the residual loss; returns the FP32 weights (device tensor) and the loss
    history.  Step t uses operator t mod len(ops) (among those with samples) and a batch of
    its samples; `select` (boolean mask over the samples) restricts the training set."""
    n, _, H, W = X.shape
    w = torch.as_tensor(he_init(seed) if w0 is None else w0, device="cuda").contiguous()
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    xd = torch.as_tensor(X, device="cuda")
    rd = torch.as_tensor(R, device="cuda")
    y = torch.empty((batch, 1, H, W), dtype=torch.float32, device="cuda")
    keep = np.ones(owner.shape, dtype=bool) if select is None else np.asarray(select, dtype=bool)
    pools = [np.nonzero((owner == o) & keep)[0] for o in range(len(ops))]
    used = [o for o in range(len(ops)) if pools[o].size > 0]
    rng = np.random.default_rng(seed + 1)
    hist = []
    for t in range(1, steps + 1):
        o = used[(t - 1) % len(used)]
        idx = torch.as_tensor(rng.choice(pools[o], size=batch), device="cuda")
        xb = xd[idx].contiguous()
        rb = rd[idx].contiguous()
        hist.append(kc_cnn_train_step_residual(ctx, w, m, v, t, lr, ops[o], xb, rb, batch,
                                               H, W, y))
    return w, hist
