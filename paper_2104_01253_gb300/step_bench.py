"""Per-step kernel times of one 50-column DCGS2 expansion, by FP64 mode.

    python -m paper_2104_01253_gb300.step_bench [--N 252] [--modes 1 2] [--steps 50]
                                                [--basis f64|f32|bf16]

The operator is the 3D convection-diffusion matrix on an N^3 grid (N = 252: m = 16,003,008,
N = 100: m = 1,000,000), start vector seed 1002.  After one untimed expansion, every step
of a second one is timed kernel by kernel with per-launch CUDA events (kc_timing_enable)
and a synchronize after the step.  Prints one JSON line per mode: the summed milliseconds
of the reduction, update and SpMV launches over the expansion, and per step k the three
times in microseconds.  FP64 modes: 0 all-FP64 products, 1 float-float offload of S and
Q C, 2 the reduction as exact digit products on the tensor cores (they apply to an FP64
basis).  --basis f32 / bf16: an FP32 or BF16 basis with FP32 vectors and an FP32 copy of
the operator (the inner solves of iterative refinement).
"""
from __future__ import annotations

import argparse
import json

import torch

from . import (KC_BF16, KC_F32, KC_F64, ArnoldiState, Context, DeviceCSR, dcgs2_arnoldi_init,
               dcgs2_arnoldi_step)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--N", type=int, default=252)
    p.add_argument("--modes", type=int, nargs="+", default=[1], choices=[0, 1, 2])
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--basis", default="f64", choices=["f64", "f32", "bf16"])
    a = p.parse_args()
    import synth
    Ah = synth.config2_operator(a.N)
    ctx = Context(0)
    qdt = {"f64": KC_F64, "f32": KC_F32, "bf16": KC_BF16}[a.basis]
    A = DeviceCSR(Ah, dtype=torch.float64 if a.basis == "f64" else torch.float32)
    st = ArnoldiState(Ah.m, a.steps + 1, qdt)
    r0 = torch.as_tensor(synth.gaussian_vector(Ah.m, 1002), device="cuda",
                         dtype=torch.float64 if a.basis == "f64" else torch.float32)
    for mode in a.modes:
        ctx.set_fp64_mode(mode)
        dcgs2_arnoldi_init(ctx, A, st, r0)
        for _ in range(a.steps):
            dcgs2_arnoldi_step(ctx, A, st)
        torch.cuda.synchronize()
        dcgs2_arnoldi_init(ctx, A, st, r0)
        torch.cuda.synchronize()
        ctx.timing_enable(True)
        ctx.timing_read()                                  # (reading clears the records)
        per_k = []
        for k in range(a.steps):
            dcgs2_arnoldi_step(ctx, A, st)
            torch.cuda.synchronize()
            d = {kk: v[0] for kk, v in ctx.timing_read().items()}
            per_k.append([k] + [round(1e3 * d.get(kk, 0.0), 1)
                                for kk in ("reduce", "dcgs2_update", "spmv")])
        ctx.timing_enable(False)
        status = ctx.read_status()
        print(json.dumps({"m": Ah.m, "basis": a.basis, "fp64_mode": mode, "status": status,
                          "ms": {kk: round(sum(r[i] for r in per_k) / 1e3, 3)
                                 for i, kk in enumerate(("reduce", "update", "spmv"), 1)},
                          "per_step_us": {"columns": ["k", "reduce", "update", "spmv"],
                                          "rows": per_k}}), flush=True)
    ctx.set_fp64_mode(1)


if __name__ == "__main__":
    main()
