"""Training the convolutional preconditioner on the GPU (orchestration of C-ABI calls).

Data: for each seeded operator of the variable-coefficient family (synth.varcoef_fields_2d),
plain DCGS2-GMRES(n) solves A x = b to 1e-10 (gmres_solve); a second run from x0 = 0,
one restart cycle per call, records every iterate x_j; each pair is the residual
r_j = b - A x_j and the correction e_j = x* - x_j (so A e_j = r_j), both divided by
rms(r_j).  The preconditioner is M(r) = r + net(r) (fgmres_solve), so the network is
trained on the target d = e - r: (1/B) sum ||net(r) - d||^2 / ||d||^2 with Adam; every
forward, backward and update runs in libkrylov (kc_cnn_train_step).
"""
from __future__ import annotations

import numpy as np
import torch

from . import (Context, DeviceCSR, gmres_solve, kc_cnn_param_count, kc_cnn_train_step,
               kc_spmv)


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


def generate_pairs(ctx: Context, N: int, seeds, restart: int = 40, max_cycles: int = 40,
                   rhs_seed_offset: int = 1000):
    """(residual, correction - residual) pairs from plain GMRES solves, scaled by
    rms(residual): the training inputs and targets of the network."""
    rs, es = [], []
    for seed in seeds:
        Ah = varcoef_operator(N, seed)
        A = DeviceCSR(Ah)
        from synth import gaussian_vector
        b = torch.as_tensor(gaussian_vector(Ah.m, rhs_seed_offset + seed), device="cuda")
        xs = torch.zeros_like(b)
        gmres_solve(ctx, A, b, xs, restart=restart, rtol=1e-10)
        x = torch.zeros_like(b)
        Ax = torch.empty_like(b)
        for _ in range(max_cycles):
            info = gmres_solve(ctx, A, b, x, restart=restart, rtol=1e-10, maxit=restart)
            kc_spmv(ctx, A, x, Ax)
            r = b - Ax
            e = xs - x
            s = torch.sqrt(torch.mean(r * r))
            if not float(s) > 0 or info["rel_resid_true"] <= 1e-9:
                break
            rs.append((r / s).float().cpu().numpy())
            es.append(((e - r) / s).float().cpu().numpy())
    r = np.stack(rs).reshape(-1, 1, N, N)
    e = np.stack(es).reshape(-1, 1, N, N)
    return r, e


def train(ctx: Context, r: np.ndarray, e: np.ndarray, steps: int = 400, batch: int = 16,
          lr: float = 1e-3, seed: int = 0, w0=None):
    """Adam on the GPU; returns the FP32 weights (device tensor) and the loss history."""
    n, _, H, W = r.shape
    w = torch.as_tensor(he_init(seed) if w0 is None else w0, device="cuda").contiguous()
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    rd = torch.as_tensor(r, device="cuda")
    ed = torch.as_tensor(e, device="cuda")
    y = torch.empty((batch, 1, H, W), dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(seed + 1)
    hist = []
    for t in range(1, steps + 1):
        idx = torch.as_tensor(rng.choice(n, size=batch, replace=n < batch), device="cuda")
        xb = rd[idx].contiguous()
        eb = ed[idx].contiguous()
        hist.append(kc_cnn_train_step(ctx, w, m, v, t, lr, xb, eb, batch, H, W, y))
    return w, hist
