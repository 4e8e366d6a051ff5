"""Time one restarted DCGS2-GMRES solve and break it down by kernel kind.

    python -m paper_2104_01253_gb300.solver_bench [--config 1|2] [--restart 30]
                                                  [--stencil] [--reps 3] [--path 0|1|2|3]
                                                  [--precision 0|1|2]

config 1: the 2D convection-diffusion operator on a 100 x 100 grid (m = 10,000), b ~ N(0,1)
seed 1001, GMRES(30); config 2: the 252^3 operator (m = 16,003,008), b seed 1004,
GMRES(50); --grid2d N: config 1's operator family on an N x N grid (b seed 1001,
GMRES(30)).  All to a relative residual of 1e-10 from x0 = 0, after one warm-up solve.
Prints one JSON line: wall time per solve (CUDA events around the C-ABI call, b and x
resident on the GPU), iterations, launches per solve, and the summed device time of each
kernel kind from a separate solve timed with per-launch CUDA events (kc_timing_enable),
whose gap to the wall time is host launch overhead and idle device time.  --path selects
the FP64 solve path (0 by size, 1 multi-kernel, 2 one thread-block cluster, 3 one CTA per
SM over the whole GPU).  --precision 1 / 2: FP32 / BF16-basis inner solves in FP64
iterative refinement (inner tolerance 1e-4, at most 3 inner cycles, as bench.py), with
an FP32 copy of the operator.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import Context, DeviceCSR, DeviceStencil7, gmres_solve


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--config", type=int, default=1, choices=[1, 2])
    p.add_argument("--restart", type=int, default=None)
    p.add_argument("--grid2d", type=int, default=None, help="N x N grid of config 1's family")
    p.add_argument("--stencil", action="store_true", help="matrix-free operator")
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--path", type=int, default=0, choices=[0, 1, 2, 3])
    p.add_argument("--precision", type=int, default=0, choices=[0, 1, 2])
    a = p.parse_args()
    import synth
    if a.grid2d:
        wind = 10.0 * np.array([1.0, 1.0]) / np.sqrt(2.0)
        op = (synth.convdiff_stencil7(a.grid2d, 2, wind) if a.stencil
              else synth.convdiff_csr(a.grid2d, 2, wind))
        seed, restart = 1001, 30
    elif a.config == 1:
        op = synth.config1_stencil() if a.stencil else synth.config1_operator()
        seed, restart = 1001, 30
    else:
        op = synth.config2_stencil() if a.stencil else synth.config2_operator()
        seed, restart = 1004, 50
    restart = a.restart or restart
    ctx = Context(0)
    ctx.set_gmres_path(a.path)
    A = DeviceStencil7(op) if a.stencil else DeviceCSR(op)
    A32 = None
    if a.precision:
        A32 = (DeviceStencil7(op, dtype=torch.float32) if a.stencil
               else DeviceCSR(op, dtype=torch.float32))
    m = A.m
    solve = lambda: gmres_solve(ctx, A, b, x, restart=restart, rtol=1e-10,
                                precision=a.precision, A32=A32, inner_rtol=1e-4,
                                inner_max_cycles=3)
    b = torch.as_tensor(synth.gaussian_vector(m, seed), device="cuda")
    x = torch.zeros_like(b)
    solve()                                                           # warm-up
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    launches0 = ctx.launch_count()
    t0.record()
    for _ in range(a.reps):
        x.zero_()
        info = solve()
    t1.record()
    torch.cuda.synchronize()
    launches = (ctx.launch_count() - launches0) // a.reps
    ms = t0.elapsed_time(t1) / a.reps
    x.zero_()
    ctx.timing_enable(True)
    solve()
    torch.cuda.synchronize()
    kinds = ctx.timing_read()
    ctx.timing_enable(False)
    print(json.dumps({"config": ("2d N=%d" % a.grid2d) if a.grid2d else a.config,
                      "operator": "stencil" if a.stencil else "csr",
                      "path": ["auto", "multi-kernel", "cluster", "grid"][a.path],
                      "precision": ["fp64", "fp32-inner-ir", "bf16-basis-ir"][a.precision],
                      "m": m, "restart": restart, "ms_per_solve": ms, "iters": info["iters"],
                      "status": info["status"], "rel_resid_true": info["rel_resid_true"],
                      "launches_per_solve": launches,
                      "us_per_iteration": 1e3 * ms / max(info["iters"], 1),
                      "device_ms_by_kind": {k: v[0] for k, v in kinds.items()},
                      "launches_by_kind": {k: v[1] for k, v in kinds.items()}}), flush=True)


if __name__ == "__main__":
    main()
