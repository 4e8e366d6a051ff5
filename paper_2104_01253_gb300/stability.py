"""Loss of orthogonality and representation error of the DCGS2 QR over condition numbers.

    python -m paper_2104_01253_gb300.stability [--m 1000000] [--n 50] [--kmax 16]
                                               [--fp64-mode 1]

Table 3 of the paper puts DCGS2 (QR) in the O(eps) loss-of-orthogonality class, with CGS2,
against O(eps) kappa for MGS and O(eps) kappa^2 for CGS.  This runs `dcgs2_qr` on seeded
graded matrices A = U diag(sigma) V^T (one pair of orthonormal factors, seed 900; sigma
log-spaced from 1 to 1/kappa) for kappa = 10^0 .. 10^kmax and prints one JSON line per
kappa: ||I - Q^T Q||_F, ||A - Q R||_F / ||A||_F, the device status and the time of the
factorisation (CUDA events around the call, A resident on the GPU).  The two norms are
evaluated with PyTorch matrix products: they measure the result, they are not part of it.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import Context, dcgs2_qr


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--m", type=int, default=1_000_000)
    p.add_argument("--n", type=int, default=50)
    p.add_argument("--kmax", type=int, default=16)
    p.add_argument("--fp64-mode", type=int, default=1, choices=[0, 1])
    a = p.parse_args()
    from synth import graded_factors, graded_matrix

    ctx = Context(0)
    ctx.set_fp64_mode(a.fp64_mode)
    m, n = a.m, a.n
    ld = m + (m & 1)
    factors = graded_factors(m, n, 900)
    At = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
    Qt = torch.zeros_like(At)
    Rt = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    for e in range(a.kmax + 1):
        B = graded_matrix(m, n, 10.0 ** e, 900, factors=factors)
        At[:, :m] = torch.as_tensor(np.ascontiguousarray(B.T), device="cuda")
        dcgs2_qr(ctx, At, Qt, Rt)                              # warm-up
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        dcgs2_qr(ctx, At, Qt, Rt)
        t1.record()
        torch.cuda.synchronize()
        status = ctx.read_status()
        Q = Qt[:, :m]
        A = At[:, :m]
        loo = torch.linalg.norm(eye - Q @ Q.T).item()
        # stored transposed: At = Rt Qt with Rt[j, i] = R(i, j)
        res = (torch.linalg.norm(A - Rt @ Q) / torch.linalg.norm(A)).item()
        print(json.dumps({"kappa": 10.0 ** e, "m": m, "n": n, "loo": loo,
                          "representation_error": res, "device_status": status,
                          "seconds": t0.elapsed_time(t1) / 1e3,
                          "fp64_mode": a.fp64_mode}), flush=True)


if __name__ == "__main__":
    main()
