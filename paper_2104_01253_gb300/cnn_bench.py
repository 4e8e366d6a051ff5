"""Time the learned preconditioner's kernels: forward passes and training steps.

    python -m paper_2104_01253_gb300.cnn_bench [--N 1024] [--batch 1] [--conv 1]
                                               [--forward 20] [--train 5]

Runs `kc_cnn_forward` and `kc_cnn_train_step` (regression loss, no Adam update) on a
seeded random batch of N x N single-channel images with He-initialised weights, after
two warm-up calls of each, and prints one JSON line with the mean time per call (CUDA
events on the current stream) and the forward pass's FLOP rate.  `--conv` selects the
kernel of the 32 -> 32 layers (0 mma.sync, 1 tcgen05).
"""
from __future__ import annotations

import argparse
import json

import torch

from . import Context, kc_cnn_forward, kc_cnn_train_step
from .train import he_init


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--N", type=int, default=1024)
    p.add_argument("--batch", type=int, default=1)
    p.add_argument("--conv", type=int, default=1, choices=[0, 1])
    p.add_argument("--forward", type=int, default=20, help="timed forward passes")
    p.add_argument("--train", type=int, default=5, help="timed training steps")
    a = p.parse_args()
    ctx = Context(0)
    ctx.set_conv_kernel(a.conv)
    B, N = a.batch, a.N
    w = torch.as_tensor(he_init(0), device="cuda")
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.randn(B, 1, N, N, device="cuda", generator=g)
    e = torch.randn(B, 1, N, N, device="cuda", generator=g)
    y = torch.empty_like(x)

    def timed(fn, reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(reps):
            fn()
        t1.record()
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / max(reps, 1)

    out = {"N": N, "batch": B, "conv": ["mma.sync", "tcgen05"][a.conv]}
    if a.forward > 0:
        ms = timed(lambda: kc_cnn_forward(ctx, w, x, y, B, N, N), a.forward)
        flop = B * N * N * (4 * 32 * 32 * 9 * 2 + 2 * 32 * 9 * 2)
        out.update(forward_ms=ms, forward_tflops=flop / ms / 1e9)
    if a.train > 0:
        wt = w.clone()
        out["train_step_ms"] = timed(
            lambda: kc_cnn_train_step(ctx, wt, None, None, 0, 0.0, x, e, B, N, N, y), a.train)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
