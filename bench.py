#!/usr/bin/env python
"""Benchmark: DCGS2 Arnoldi-QR throughput on the 252^3 convection-diffusion operator.

One benchmark "step" is one full Arnoldi expansion of n = 50 columns through the C ABI:
init (w = r0), 50 DCGS2 steps (SpMV + one fused reduction with the scalar step + fused
update each) and the CGS2 finish.  The reported metric is Arnoldi steps (basis columns)
per second; HBM GB/s (algorithmic bytes) is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Measurement suites (one GPU, one JSON line each; not the benchmark line):
  python bench.py --suite steps  [--N 252] [--n 50] [--modes 1 2] [--basis f64|f32|bf16]
      per-step kernel times of one expansion (reduction, update, SpMV), by FP64 mode;
  python bench.py --suite solver [--config 1|2] [--grid2d N] [--path 0..3] [--precision 0..2]
                                 [--matrix-free] [--restart n] [--reps 3]
      one restarted GMRES solve to 1e-10, wall time and device time by kernel kind;
  python bench.py --suite cnn    [--N 1024] [--batch 1] [--conv 0|1] [--forward 20] [--train 5]
      the learned preconditioner's forward pass and training step;
  python bench.py --suite learn  [--N 1024]
      config 5 as a study: learning curve, held-out operators 64-71, extrapolated baselines;
  python bench.py --suite part   [--N 252] [--n 50]
      the row-partitioned expansion with P = 1, 2, 4 ranks emulated on one GPU.

Under torchrun each rank runs an independent replica of the workload on its own GPU
(weak scaling, no data-path collective); rank 0 prints one JSON line.  The reference arm
(--impl reference) times the FP64 CPU oracle on the host cores on a bounded sample of
the same workload, scaled to the metric's unit.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import config2_operator, config2_stencil, convdiff_csr, gaussian_vector  # noqa: E402

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# FP64 FMA peak derived from unit counts and the maximum clock: 152 SMs x 2 DFMA/clk/SM
# x 2 flop x 2.070 GHz (a DFMA throughput probe measured 1.20 TFLOP/s at 2.0 GHz)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# DRAM bytes (read + write) over algorithmic bytes of the offload-mode register-streaming
# kernels, from the ncu capture summarised in profiles/launches_dcgs2_m16003008_n50.md
# (steps k = 25 and 26 at m = 4,096,000).  Valid only for those kernels as captured.
TRAFFIC_RATIO = {"reduce": 1.007, "dcgs2_update": 0.950}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--N", type=int, default=252, help="grid points per direction (m = N^3)")
    p.add_argument("--n", type=int, default=50, help="Arnoldi steps per expansion")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-baselines", action="store_true")
    p.add_argument("--no-stencil", action="store_true",
                   help="skip the matrix-free stencil expansions and solves")
    p.add_argument("--no-solvers", action="store_true",
                   help="skip the GMRES time-to-1e-10 runs (plain FP64 vs FP32/BF16 IR)")
    p.add_argument("--fp64-mode", type=int, default=1, choices=[0, 1, 2])
    p.add_argument("--staged", type=int, default=None, choices=[0, 1, 2, 3, 8],
                   help="kernel variants of the basis passes (kc_set_staged flags); "
                        "default: the library's")
    p.add_argument("--no-check", action="store_true",
                   help="skip the loss-of-orthogonality / Arnoldi-relation check")
    p.add_argument("--suite", default=None,
                   choices=["steps", "solver", "cnn", "learn", "part"],
                   help="a measurement suite instead of the benchmark line (module docstring)")
    p.add_argument("--modes", type=int, nargs="+", default=[1], choices=[0, 1, 2])
    p.add_argument("--basis", default="f64", choices=["f64", "f32", "bf16"])
    p.add_argument("--config", type=int, default=1, choices=[1, 2])
    p.add_argument("--grid2d", type=int, default=None)
    p.add_argument("--path", type=int, default=0, choices=[0, 1, 2, 3])
    p.add_argument("--precision", type=int, default=0, choices=[0, 1, 2])
    p.add_argument("--matrix-free", action="store_true")
    p.add_argument("--restart", type=int, default=None)
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--batch", type=int, default=1)
    p.add_argument("--conv", type=int, default=1, choices=[0, 1])
    p.add_argument("--forward", type=int, default=20)
    p.add_argument("--train", type=int, default=5)
    p.add_argument("--no-parity", action="store_true",
                   help="skip the full-size comparison of H and sampled Q rows with the FP64 "
                        "oracle (about a minute of host time, outside the timed region)")
    return p.parse_args()


def algorithmic_bytes(m, nnz, n):
    """HBM bytes of one expansion (n DCGS2 steps + finish), FP64, int32 indices.

    step k: SpMV 4(m+1) + 12 nnz + 8m (x) + 8m (y); reduction 8mk + 16m (Q_k, w, v);
    update 8mk + 16m reads + 16m writes (q_k, w).  finish, counted as the method's CGS2
    pass (two projections' sums and two projections, whatever the kernels fuse):
    2*(8mk + 8m) + 2*(8mk + 16m), norm 8m, scaling 16m.  The steps alone are 16mk + 48m
    plus the SpMV each; the fused passes (the first steps' SpMV with
    the reduction, the finish's u = w - Q C1 with the second projection's sums) move less
    than this count."""
    spmv = 4 * (m + 1) + 12 * nnz + 16 * m
    total = 0
    per_kernel = {"spmv": 0, "reduce": 0, "dcgs2_update": 0}
    for k in range(n):
        per_kernel["spmv"] += spmv
        per_kernel["reduce"] += 8 * m * k + 16 * m
        per_kernel["dcgs2_update"] += 8 * m * k + 32 * m
    k = n
    fin = 2 * (8 * m * k + 8 * m) + 2 * (8 * m * k + 16 * m) + 8 * m + 16 * m
    total = sum(per_kernel.values()) + fin
    return total, per_kernel


def kernel_rooflines(kern, m, nnz, n, steps, fp64_mode, hbm_peak):
    """Achieved rates of the step's kernels from their CUDA-event times (kc_timing_read):
    algorithmic bytes and FLOPs per expansion (the n DCGS2 steps) over each kernel's summed
    launch time.  Reduction at step k: bytes 8 m k + 16 m (Q_k, w, v); FP64-pipe FMAs
    m k f (+ 2 m for beta and s in the all-FP64 mode; with offload the SpMV forms them) with
    f = 1 with offload, 2 all-FP64, against the method's 2 m k + 2 m.  Update:
    bytes 8 m k + 32 m; FP64-pipe operations m k f + 3 m (v / alpha, q and w' per row)
    against 2 m k + 3 m.  SpMV: 4 (m + 1) + 12 nnz + 16 m bytes, nnz + 2 m FMAs (the matvec,
    beta and s).  With the first steps fused (flag 8, k <= 4: `spmv_reduce`) those steps
    count under that kind, with the SpMV's bytes plus 8 m k and its FMAs plus m k, and the
    SpMV and reduction rows cover the other steps.  The CGS2 finish (k = n): the first
    projection's sums (8 m k + 8 m bytes;
    with offload its column sums are float-float, so m FP64 FMAs for x^T x, else m k + m) and
    the fused u = w - Q C1 with the second projection's sums (8 m k + 16 m bytes, m k + m
    FMAs).  In FP64 mode 2
    the reduction's products are exact integer digit products on the tensor cores (no FP64
    FMA per element)."""
    f = 2 if fp64_mode == 0 else 1
    fr = {0: 2, 1: 1, 2: 0}[fp64_mode]            # mode 2: the reduction has no FP64 FMA
    bs = 2 if fp64_mode == 0 else 0               # beta, s FMAs per row in the reduction
    # with kc_set_staged flag 8 the first nf steps (FP64 mode 1) form v = A w and the
    # reduction in one fused pass:
    # the SpMV's bytes plus the basis columns (w and v are not read again), the SpMV's FMAs
    # plus m k for C (S is float-float)
    nf = kern.get("spmv_reduce", (0.0, 0))[1] // max(steps, 1)
    sp = 4 * (m + 1) + 12 * nnz + 16 * m
    rows = {
        "reduce": (sum(8 * m * k + 16 * m for k in range(nf, n)),
                   sum(m * k * fr + bs * m for k in range(nf, n)),
                   sum(2 * m * k + 2 * m for k in range(nf, n)), n - nf),
        "dcgs2_update": (sum(8 * m * k + 32 * m for k in range(n)),
                         sum(m * k * f + 3 * m for k in range(n)),
                         sum(2 * m * k + 3 * m for k in range(n)), n),
        "spmv": ((n - nf) * sp, (n - nf) * (nnz + 2 * m), (n - nf) * (nnz + 2 * m), n - nf),
        "spmv_reduce": (sum(sp + 8 * m * k for k in range(nf)),
                        sum(nnz + 2 * m + m * k for k in range(nf)),
                        sum(nnz + 2 * m + 2 * m * k for k in range(nf)), nf),
        "finish_reduce": ((8 * m * n + 8 * m) + (8 * m * n + 16 * m),
                          (m if fp64_mode >= 1 else m * n + m) + (m * n + m),
                          2 * (m * n + m), 2),
    }
    out = {}
    for name, (byts, fma_pipe, fma_method, launches) in rows.items():
        ms_k, cnt_k = kern.get(name, (0.0, 0))
        if cnt_k == 0 or ms_k <= 0.0 or launches == 0:
            continue
        t = ms_k / 1e3
        tf = 2.0 * fma_pipe * steps / t / 1e12
        gbs = byts * steps / t / 1e9
        out[name] = {"ms_per_step": ms_k / steps, "launches": cnt_k,
                     "avg_launch_ms": ms_k / cnt_k, "bytes_per_launch": byts / launches,
                     "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak,
                     "fp64_tflops": tf, "fp64_frac": tf / FP64_PEAK_TFLOPS,
                     "method_tflops": 2.0 * fma_method * steps / t / 1e12,
                     "fp64_fma_per_elem": (fr if name == "reduce" else
                                           (f if name == "dcgs2_update" else None))}
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if not self.samples:
            return None
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device: str = "cuda") -> float:
    """The largest value of x over all ranks (the slowest rank's time); x itself at ws = 1.
    The process group's backend decides the device of the exchanged tensor (NCCL: cuda)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(ws: int, n: int, steps: int, ms_max: float) -> float:
    """Whole-job Arnoldi steps per second: every rank ran `steps` expansions of n steps,
    timed by the slowest rank."""
    return ws * n * steps / (ms_max / 1e3)


def cpu_oracle_sample(n, N_sample=126, seed=1002):
    """Time the FP64 oracle on one full n-step expansion of the same operator family at
    N_sample^3 rows; returns (steps/s scaled to the full-size m, seconds, m_sample)."""
    from oracle import arnoldi as orc
    Ah = convdiff_csr(N_sample, 3, 50.0 * np.array([1.0, 0.5, 0.25]) / np.linalg.norm([1.0, 0.5, 0.25]))
    A = Ah.to_scipy()
    r0 = gaussian_vector(Ah.m, seed)
    t0 = time.perf_counter()
    orc.dcgs2_arnoldi(A, r0, n)
    dt = time.perf_counter() - t0
    return n / dt, dt, Ah.m


def full_size_parity(Ah, r0, n, H_gpu, q_rows, Q_gpu):
    """The timed expansion against the FP64 oracle at the benchmark's own size (outside the
    timed region): ||H - H_o||_F / ||H_o||_F and the largest error over sampled rows of
    Q, with the benchmark spec's tolerances 1e-12 and 1e-10."""
    from oracle import arnoldi as orc
    t0 = time.perf_counter()
    Qo, Ho = orc.dcgs2_arnoldi(Ah.to_scipy(), r0, n)
    dt = time.perf_counter() - t0
    herr = float(np.linalg.norm(H_gpu - Ho) / np.linalg.norm(Ho))
    qerr = float(np.abs(Q_gpu - Qo[q_rows]).max())
    col = np.linalg.norm(H_gpu - Ho, axis=0) / np.maximum(np.linalg.norm(Ho, axis=0), 1e-300)
    return {"H_rel_frobenius": herr, "H_worst_column_rel": float(col.max()),
            "Q_sampled_rows": int(len(q_rows)), "Q_max_abs": qerr,
            "pass": bool(herr <= 1e-12 and qerr <= 1e-10), "oracle_seconds": dt,
            "tolerances": {"H_rel": 1e-12, "Q_abs": 1e-10}}


def quality(kc, ctx, A, st, m, n):
    """||I - Q^T Q||_F and ||A Q_n - Q_{n+1} H||_F / ||A||_F of the last expansion
    (check only; uses torch matmuls outside the timed region)."""
    import torch
    Qv = st.Qbuf[:n + 1, :m]
    G = Qv @ Qv.T
    loo = float(torch.linalg.norm(torch.eye(n + 1, device="cuda", dtype=torch.float64) - G))
    H = st.Hbuf[:n, :n + 1].T.contiguous()
    AQ = torch.empty(n, m, dtype=torch.float64, device="cuda")
    for j in range(n):
        kc.kc_spmv(ctx, A, Qv[j], AQ[j])
    R = AQ - (H.T @ Qv)
    rre = float(torch.linalg.norm(R)) / float(torch.linalg.norm(A.val))
    return loo, rre


def solver_suite(kc, ctx, A, m, stream):
    """GMRES time to a 1e-10 relative residual, measured with CUDA events around the
    C-ABI call (device-resident b and x): config 1 (2D, 100^2, GMRES(30)) and, on the
    config-2 matrix, plain FP64 DCGS2-GMRES(50) against FP32- and BF16-basis GMRES(50)
    inner solves in FP64 iterative refinement (b ~ N(0,1), seed 1004); the DCGS2 QR of an
    m x 50 matrix; the learned preconditioner (config-5 family)."""
    import torch
    from synth import config1_operator
    from synth import config2_operator  # noqa: F401  (same operator as A)

    def timed_solve(fn):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        info = fn()
        t1.record(stream)
        torch.cuda.synchronize()
        info["seconds"] = t0.elapsed_time(t1) / 1e3
        return info

    out = {}
    A1h = config1_operator()
    A1 = kc.DeviceCSR(A1h)
    b1 = torch.as_tensor(gaussian_vector(A1h.m, 1001), device="cuda")
    x1 = torch.zeros_like(b1)
    kc.gmres_solve(ctx, A1, b1, x1, restart=30, rtol=1e-10)          # warm-up
    x1.zero_()
    out["config1_fp64_gmres30"] = timed_solve(
        lambda: kc.gmres_solve(ctx, A1, b1, x1, restart=30, rtol=1e-10))
    out["config1_fp64_gmres30"]["path"] = "one launch, one CTA per SM (grid barrier)"
    for name, path in (("config1_fp64_gmres30_cluster", ctx.GMRES_CLUSTER),
                       ("config1_fp64_gmres30_multi_kernel", ctx.GMRES_MULTI_KERNEL)):
        ctx.set_gmres_path(path)
        x1.zero_()
        kc.gmres_solve(ctx, A1, b1, x1, restart=30, rtol=1e-10)       # warm-up
        x1.zero_()
        out[name] = timed_solve(lambda: kc.gmres_solve(ctx, A1, b1, x1, restart=30, rtol=1e-10))
    ctx.set_gmres_path(ctx.GMRES_AUTO)
    A32 = kc.DeviceCSR.__new__(kc.DeviceCSR)
    A32.m, A32.nnz = A.m, A.nnz
    A32.row_ptr, A32.col_idx = A.row_ptr, A.col_idx
    A32.val = A.val.float()
    A32.val_dtype = kc.KC_F32
    A32.c = kc.kc_csr(A32.m, A32.nnz, A32.row_ptr.data_ptr(), A32.col_idx.data_ptr(),
                      A32.val.data_ptr(), kc.KC_F32)
    b = torch.as_tensor(gaussian_vector(m, 1004), device="cuda")
    for name, prec in (("config4_fp64_gmres50", 0), ("config4_ir_fp32_gmres50", 1),
                       ("config4_ir_bf16basis_gmres50", 2)):
        x = torch.zeros_like(b)
        out[name] = timed_solve(lambda: kc.gmres_solve(
            ctx, A, b, x, restart=50, rtol=1e-10, precision=prec, A32=A32, inner_rtol=1e-4,
            inner_max_cycles=3))
    # accuracy of each config-4 solve: the worst loss of orthogonality of its (inner)
    # bases, from a second run with the diagnostic on (not timed)
    for name, prec in (("config4_fp64_gmres50", 0), ("config4_ir_fp32_gmres50", 1),
                       ("config4_ir_bf16basis_gmres50", 2)):
        x = torch.zeros_like(b)
        d = kc.gmres_solve(ctx, A, b, x, restart=50, rtol=1e-10, precision=prec, A32=A32,
                           inner_rtol=1e-4, inner_max_cycles=3, diag_loo=True)
        out[name]["max_loo_over_cycles"] = d["max_loo"]
    del A32
    out["config4_accuracy_64cubed"] = config4_accuracy(kc, ctx)
    out.update(qr_suite(kc, ctx, m, stream))
    out.update(ks_suite(kc, ctx, timed_solve))
    out.update(learned_suite(kc, ctx, timed_solve))
    return out


def config4_accuracy(kc, ctx, N=64):
    """Solution error of the three config-4 solvers against the FP64 oracle's own
    DCGS2-GMRES(50) solution on the same operator family at N^3 rows (the oracle finishes
    there in seconds; at 252^3 it would take minutes), with the same b recipe (seed 1004):
    ||x - x_o|| / ||x_o||, the true residual and the worst loss of orthogonality of the
    (inner) bases.  Two solves that each reach 1e-10 differ by up to about kappa(A) 1e-10
    (reading 13), so the error is reported next to both residuals."""
    import torch
    from oracle.gmres import gmres as orc_gmres
    Ah = config2_operator(N)
    A = kc.DeviceCSR(Ah)
    A32 = kc.DeviceCSR(Ah, dtype=torch.float32)
    bh = gaussian_vector(Ah.m, 1004)
    t0 = time.perf_counter()
    xo, io = orc_gmres(Ah.to_scipy(), bh, restart=50, rtol=1e-10)
    out = {"m": Ah.m, "oracle": {"iters": io["iters"], "rel_resid_true": io["rel_resid_true"],
                                 "seconds": time.perf_counter() - t0}}
    b = torch.as_tensor(bh, device="cuda")
    for name, prec in (("fp64_gmres50", 0), ("ir_fp32_gmres50", 1), ("ir_bf16basis_gmres50", 2)):
        x = torch.zeros_like(b)
        info = kc.gmres_solve(ctx, A, b, x, restart=50, rtol=1e-10, precision=prec, A32=A32,
                              inner_rtol=1e-4, inner_max_cycles=3, diag_loo=True)
        xh = x.cpu().numpy()
        out[name] = {"iters": info["iters"], "outer": info["outer"],
                     "rel_resid_true": info["rel_resid_true"],
                     "rel_error_vs_oracle": float(np.linalg.norm(xh - xo) / np.linalg.norm(xo)),
                     "max_loo_over_cycles": info["max_loo"], "status": info["status"]}
    return out


def ks_suite(kc, ctx, timed_solve):
    """Krylov-Schur on config 3 (2D, N = 1000, m = 10^6, kappa i.i.d. log-uniform on
    [0.1, 10], seed 1003; start vector seed 1003): the 10 eigenvalues of largest real part
    with 40-column expansions restarted to 20, to a relative Ritz residual of 1e-10 (the
    eigenvalues themselves are checked against dense eigenvalues on the 40 x 40 copy by
    the tests).  Time by CUDA events around the C-ABI call, after a one-restart warm-up."""
    import torch
    from synth import config3_operator
    A3h = config3_operator()
    A3 = kc.DeviceCSR(A3h)
    v0 = torch.as_tensor(gaussian_vector(A3h.m, 1003), device="cuda")
    del A3h
    kc.krylov_schur_eigs(ctx, A3, v0, nev=10, ncv=40, nkeep=20, tol=1e-10, maxrestarts=1)
    res = timed_solve(lambda: kc.krylov_schur_eigs(ctx, A3, v0, nev=10, ncv=40, nkeep=20,
                                                   tol=1e-10, maxrestarts=2000))
    eigs = res.pop("eigs")
    resid = res.pop("resid")
    res["max_rel_ritz_residual"] = float(np.max(resid / np.maximum(np.abs(eigs), 1e-300)))
    res["eigs_largest_real"] = [[float(z.real), float(z.imag)] for z in eigs]
    return {"config3_krylov_schur_nev10_ncv40": res}


def qr_suite(kc, ctx, m, stream, n=50, reps=3):
    """DCGS2 QR (Algorithm 2) of an m x n matrix of seeded N(0,1) entries generated on the
    GPU (torch, seed 2021): columns per second, algorithmic HBM bytes per second and the
    loss of orthogonality of Q.  Algorithmic bytes per column k < n - 1: reduction
    8 m k + 16 m (Q_k, w, a_{k+1}), update 8 m k + 32 m (Q_k, w, a_{k+1} read; q_k, w
    written); the CGS2 finish: 2 (8 m k + 8 m) + 2 (8 m k + 16 m) + 8 m + 16 m at k = n - 1."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(2021)
    ld = m + (m & 1)
    A = torch.randn((n, ld), dtype=torch.float64, device="cuda", generator=g)
    Q = torch.empty_like(A)
    R = torch.empty((n, n), dtype=torch.float64, device="cuda")
    kc.dcgs2_qr(ctx, A, Q, R)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(reps):
        kc.dcgs2_qr(ctx, A, Q, R)
    t1.record(stream)
    torch.cuda.synchronize()
    sec = t0.elapsed_time(t1) / 1e3 / reps
    byts = sum(16 * m * k + 48 * m for k in range(n - 1))
    k = n - 1
    byts += 2 * (8 * m * k + 8 * m) + 2 * (8 * m * k + 16 * m) + 8 * m + 16 * m
    Qv = Q[:, :m]
    loo = float(torch.linalg.norm(torch.eye(n, device="cuda", dtype=torch.float64) - Qv @ Qv.T))
    res = float(torch.linalg.norm(A[:, :m] - R @ Qv) / torch.linalg.norm(A[:, :m]))
    status = ctx.read_status()
    del A, Q, R
    return {"dcgs2_qr_m%d_n%d" % (m, n): {
        "seconds": sec, "columns_per_s": n / sec, "hbm_gbs": byts / sec / 1e9,
        "algorithmic_bytes": byts, "loo": loo, "rel_residual_A_minus_QR": res,
        "device_status": status}}


def learned_suite(kc, ctx, timed_solve):
    """Config-5 family (2D variable coefficients, kappa log-normal, random smooth wind):
    the network is trained on the GPU from restart residuals of plain GMRES(40) on seeded
    operators, then plain GMRES(40), FGMRES(40) with the Jacobi step alone and FGMRES(40)
    with the learned preconditioner solve held-out operator 64 to 1e-10.  256^2: every
    method converges; 1024^2 (the config-5 grid): plain and Jacobi stop at an iteration
    cap.  Training time (data generation + 600 Adam steps) is reported separately."""
    import torch
    from paper_2104_01253_gb300 import train as tr
    out = {}
    for N, nops, cycles, batch, cap in ((256, 12, 20, 4, 40000), (1024, 16, 10, 2, 20000)):
        t0 = time.time()
        host_ops = [tr.varcoef_operator(N, seed) for seed in range(nops)]    # synthetic inputs
        setup_s = time.time() - t0
        t0 = time.time()
        ops, X, R, owner = tr.generate_pairs(ctx, N, range(nops), restart=40, max_cycles=cycles,
                                             host_ops=host_ops)
        npairs = int(X.shape[0])
        torch.cuda.synchronize()
        pairs_s = time.time() - t0
        t0 = time.time()
        w, hist = tr.train(ctx, ops, X, R, owner, steps=600, batch=batch, lr=2e-3, seed=0)
        torch.cuda.synchronize()
        train_s = time.time() - t0
        del host_ops
        del X, R, ops
        Ah = tr.varcoef_operator(N, 64)
        A = kc.DeviceCSR(Ah)
        b = torch.as_tensor(gaussian_vector(Ah.m, 2064), device="cuda")
        res = {"grid": "%d^2" % N, "training": {"operators": nops, "pairs": npairs,
                                                "adam_steps": 600, "batch": batch,
                                                "host_operator_setup_seconds": setup_s,
                                                "pair_generation_seconds": pairs_s,
                                                "seconds": train_s,
                                                "loss_first": float(np.mean(hist[:20])),
                                                "loss_last": float(np.mean(hist[-50:]))}}
        for name, fn in (
                ("plain_gmres40", lambda x: kc.gmres_solve(ctx, A, b, x, restart=40,
                                                           rtol=1e-10, maxit=cap)),
                ("jacobi_fgmres40", lambda x: kc.fgmres_solve(ctx, A, None, N, N, b, x,
                                                              restart=40, rtol=1e-10,
                                                              maxit=cap,
                                                              precond=kc.PREC_JACOBI)),
                ("learned_fgmres40", lambda x: kc.fgmres_solve(ctx, A, w, N, N, b, x,
                                                               restart=40, rtol=1e-10,
                                                               maxit=40000))):
            x = torch.zeros_like(b)
            info = timed_solve(lambda: fn(x))
            info["converged"] = info["rel_resid_true"] <= 1e-10
            res[name] = info
        out["config5_learned_%d" % N] = res
        del A, b, w
    return out


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return max(int(i.get("num_threads", 1)) for i in info)
    except Exception:
        pass
    return os.cpu_count()


def run_reference(args, ws, rank):
    if rank != 0:
        return
    m_full = args.N ** 3
    vals = []
    for i in range(args.warmup + args.steps):
        rate, dt, m_s = cpu_oracle_sample(args.n, N_sample=100)
        if i >= args.warmup:
            vals.append(rate * m_s / m_full)
    v = float(np.mean(vals))
    cores = blas_threads()
    sample = ("FP64 oracle (numpy/scipy), one %d-step DCGS2 expansion of the same operator "
              "family at 100^3 rows per step, rate scaled by rows to m = %d" % (args.n, m_full))
    line = {"impl": "reference", "metric": "arnoldi_steps_per_s", "value": v,
            "unit": "steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "dcgs2_arnoldi m=%d n=%d (3D convection-diffusion %d^3, Pe 50)"
                       % (m_full, args.n, args.N)},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def suite_steps(args):
    """Per-step kernel times of one n-step DCGS2 expansion of the N^3 operator (start vector
    seed 1002): after one untimed expansion, every step of a second one is timed kernel by
    kernel with per-launch CUDA events and a synchronize after the step."""
    import torch
    import paper_2104_01253_gb300 as kc
    import synth
    Ah = synth.config2_operator(args.N)
    ctx = kc.Context(0)
    qdt = {"f64": kc.KC_F64, "f32": kc.KC_F32, "bf16": kc.KC_BF16}[args.basis]
    fdt = torch.float64 if args.basis == "f64" else torch.float32
    A = kc.DeviceCSR(Ah, dtype=fdt)
    st = kc.ArnoldiState(Ah.m, args.n + 1, qdt)
    r0 = torch.as_tensor(synth.gaussian_vector(Ah.m, 1002), device="cuda", dtype=fdt)
    if args.staged is not None:
        ctx.set_staged(args.staged)
    for mode in args.modes:
        ctx.set_fp64_mode(mode)
        kc.dcgs2_arnoldi_init(ctx, A, st, r0)
        for _ in range(args.n):
            kc.dcgs2_arnoldi_step(ctx, A, st)
        kc.dcgs2_arnoldi_init(ctx, A, st, r0)
        torch.cuda.synchronize()
        ctx.timing_enable(True)
        ctx.timing_read()
        per_k = []
        for k in range(args.n):
            kc.dcgs2_arnoldi_step(ctx, A, st)
            torch.cuda.synchronize()
            d = {kk: v[0] for kk, v in ctx.timing_read().items()}
            per_k.append([k] + [round(1e3 * d.get(kk, 0.0), 1)
                                for kk in ("reduce", "dcgs2_update", "spmv", "spmv_reduce")])
        ctx.timing_enable(False)
        print(json.dumps({"suite": "steps", "m": Ah.m, "basis": args.basis, "fp64_mode": mode,
                          "status": ctx.read_status(),
                          "ms": {kk: round(sum(r[i] for r in per_k) / 1e3, 3)
                                 for i, kk in enumerate(("reduce", "update", "spmv",
                                                         "spmv_reduce"), 1)},
                          "per_step_us": {"columns": ["k", "reduce", "update", "spmv",
                                                      "spmv_reduce"],
                                          "rows": per_k}}), flush=True)
    ctx.set_fp64_mode(1)


def suite_solver(args):
    """One restarted DCGS2-GMRES solve to 1e-10 from x0 = 0 after a warm-up solve: config 1
    (100^2, b seed 1001, GMRES(30)), config 2 (252^3, b seed 1004, GMRES(50)) or config 1's
    family on an N x N grid; wall time (CUDA events around the C-ABI call, b and x resident)
    and, from a separate solve, device time by kernel kind."""
    import torch
    import paper_2104_01253_gb300 as kc
    import synth
    if args.grid2d:
        wind = 10.0 * np.array([1.0, 1.0]) / np.sqrt(2.0)
        op = (synth.convdiff_stencil7(args.grid2d, 2, wind) if args.matrix_free
              else synth.convdiff_csr(args.grid2d, 2, wind))
        seed, restart = 1001, 30
    elif args.config == 1:
        op = synth.config1_stencil() if args.matrix_free else synth.config1_operator()
        seed, restart = 1001, 30
    else:
        op = synth.config2_stencil() if args.matrix_free else synth.config2_operator()
        seed, restart = 1004, 50
    restart = args.restart or restart
    ctx = kc.Context(0)
    ctx.set_gmres_path(args.path)
    mk = kc.DeviceStencil7 if args.matrix_free else kc.DeviceCSR
    A = mk(op)
    A32 = mk(op, dtype=torch.float32) if args.precision else None
    b = torch.as_tensor(synth.gaussian_vector(A.m, seed), device="cuda")
    x = torch.zeros_like(b)
    solve = lambda: kc.gmres_solve(ctx, A, b, x, restart=restart, rtol=1e-10,
                                   precision=args.precision, A32=A32, inner_rtol=1e-4,
                                   inner_max_cycles=3)
    solve()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    launches0 = ctx.launch_count()
    t0.record()
    for _ in range(args.reps):
        x.zero_()
        info = solve()
    t1.record()
    torch.cuda.synchronize()
    launches = (ctx.launch_count() - launches0) // args.reps
    ms = t0.elapsed_time(t1) / args.reps
    x.zero_()
    ctx.timing_enable(True)
    solve()
    torch.cuda.synchronize()
    kinds = ctx.timing_read()
    ctx.timing_enable(False)
    print(json.dumps({"suite": "solver",
                      "config": ("2d N=%d" % args.grid2d) if args.grid2d else args.config,
                      "operator": "stencil" if args.matrix_free else "csr",
                      "path": ["auto", "multi-kernel", "cluster", "grid"][args.path],
                      "precision": ["fp64", "fp32-inner-ir", "bf16-basis-ir"][args.precision],
                      "m": A.m, "restart": restart, "ms_per_solve": ms, "iters": info["iters"],
                      "status": info["status"], "rel_resid_true": info["rel_resid_true"],
                      "launches_per_solve": launches,
                      "us_per_iteration": 1e3 * ms / max(info["iters"], 1),
                      "device_ms_by_kind": {k: v[0] for k, v in kinds.items()},
                      "launches_by_kind": {k: v[1] for k, v in kinds.items()}}), flush=True)


def suite_learn(args):
    """Config 5 as a study (one-off costs, not the step benchmark): a learning curve of the
    learned preconditioner on the N x N variable-coefficient family (default 1024^2).
    Restart residuals of plain GMRES(40) on seeded operators 0..63 (up to 160 cycles each,
    kept on the device) give three nested training sets: the first 10 cycles of operators
    0..15, the first 20 of 0..63, and all of them.  Each set trains a network from the same
    initial weights (Adam, batch 4), which then solves the held-out operators 64..71 with
    FGMRES(40) to 1e-10.  Plain GMRES(40) and FGMRES(40) with the Jacobi step alone run
    20,000 iterations on the same operators; their relative residuals after 10,000 and
    20,000 iterations give a geometric rate per iteration, from which the iterations (and
    time, at the measured time per iteration) to 1e-10 are extrapolated.  Every solve is
    timed with CUDA events around the C-ABI call; the training set sizes and all generation
    and training times are reported."""
    import torch
    import paper_2104_01253_gb300 as kc
    from paper_2104_01253_gb300 import train as tr
    from synth import gaussian_vector
    N = 1024 if args.N == 252 else args.N
    ctx = kc.Context(0)
    stream = torch.cuda.current_stream()

    def timed(fn):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        info = fn()
        t1.record(stream)
        torch.cuda.synchronize()
        info["seconds"] = t0.elapsed_time(t1) / 1e3
        return info

    out = {"suite": "learn", "grid": "%d^2" % N}
    t0 = time.time()
    host_ops = [tr.varcoef_operator(N, seed) for seed in range(64)]
    out["host_operator_setup_seconds"] = time.time() - t0
    torch.cuda.synchronize()
    t0 = time.time()
    ops, X, R, owner = tr.generate_pairs(ctx, N, range(64), restart=40, max_cycles=160,
                                         host_ops=host_ops, on_device=True)
    torch.cuda.synchronize()
    out["pair_generation_seconds"] = time.time() - t0
    out["pairs_generated"] = int(owner.size)
    del host_ops
    cycle = np.zeros(owner.size, dtype=np.int64)
    for o in range(64):
        idx = np.nonzero(owner == o)[0]
        cycle[idx] = np.arange(idx.size)
    held = list(range(64, 72))
    held_ops = [kc.DeviceCSR(tr.varcoef_operator(N, s)) for s in held]
    rhs = [torch.as_tensor(gaussian_vector(N * N, 2000 + s), device="cuda") for s in held]
    curve = []
    for nops, ncyc, steps in ((16, 10, 600), (64, 20, 1500), (64, 160, 4000)):
        sel = (owner < nops) & (cycle < ncyc)
        torch.cuda.synchronize()
        t0 = time.time()
        w, hist = tr.train(ctx, ops, X, R, owner, steps=steps, batch=4, lr=2e-3, seed=0,
                           select=sel)
        torch.cuda.synchronize()
        point = {"operators": nops, "cycles_per_operator": ncyc, "pairs": int(sel.sum()),
                 "adam_steps": steps, "batch": 4, "training_seconds": time.time() - t0,
                 "loss_first": float(np.mean(hist[:20])),
                 "loss_last": float(np.mean(hist[-50:])), "held_out": []}
        for s, A, b in zip(held, held_ops, rhs):
            x = torch.zeros_like(b)
            info = timed(lambda: kc.fgmres_solve(ctx, A, w, N, N, b, x, restart=40,
                                                 rtol=1e-10, maxit=40000))
            point["held_out"].append({"seed": s, "iters": info["iters"],
                                      "rel_resid_true": info["rel_resid_true"],
                                      "seconds": info["seconds"]})
        its = [h["iters"] for h in point["held_out"]]
        point["iters_mean"] = float(np.mean(its))
        point["seconds_mean"] = float(np.mean([h["seconds"] for h in point["held_out"]]))
        curve.append(point)
        del w
    out["curve"] = curve
    base = []
    for s, A, b in zip(held, held_ops, rhs):
        row = {"seed": s}
        for name, fn in (
                ("plain_gmres40", lambda x: kc.gmres_solve(ctx, A, b, x, restart=40,
                                                           rtol=1e-10, maxit=10000)),
                ("jacobi_fgmres40", lambda x: kc.fgmres_solve(ctx, A, None, N, N, b, x,
                                                              restart=40, rtol=1e-10,
                                                              maxit=10000,
                                                              precond=kc.PREC_JACOBI))):
            x = torch.zeros_like(b)
            a = timed(lambda: fn(x))          # restarted: the second call continues the first
            c = timed(lambda: fn(x)) if a["rel_resid_true"] > 1e-10 else None
            r10, it10 = a["rel_resid_true"], a["iters"]
            ent = {"iters": it10, "rel_resid": r10, "seconds": a["seconds"]}
            if c is not None:
                r20, it = c["rel_resid_true"], it10 + c["iters"]
                sec = a["seconds"] + c["seconds"]
                ent.update(iters=it, rel_resid=r20, seconds=sec, rel_resid_at_10000=r10)
                rate = (np.log(r20) - np.log(r10)) / max(c["iters"], 1)
                if r20 <= 1e-10:
                    ent["converged"] = True
                elif rate < 0:
                    est = it + (np.log(1e-10) - np.log(r20)) / rate
                    ent.update({"converged": False,
                                "extrapolated_iters_to_1e-10": float(est),
                                "extrapolated_seconds_to_1e-10": float(est * sec / it)})
                else:
                    ent.update(converged=False, stagnated=True)
            else:
                ent["converged"] = True
            row[name] = ent
        base.append(row)
    out["baselines"] = base
    print(json.dumps(out), flush=True)


def suite_part(args):
    """The row-partitioned DCGS2 expansion (Section 5's layout) with P ranks emulated on one
    GPU: each rank has its own context, rows of A (columns re-based onto its halo-extended
    range of w), basis rows and state; per step every rank runs dcgs2_part_reduce on its
    halo-extended w, the partial sums are added on the device (standing in for the
    all-reduce), and every rank runs dcgs2_part_update.  The ranks' kernels are timed with
    per-launch CUDA events (the halo assembly and the sum are PyTorch copies outside that
    time).  Reported per P: each rank's kernel time per expansion and their maximum, which
    is the P-GPU expansion time without communication, against the unpartitioned step."""
    import torch
    import paper_2104_01253_gb300 as kc
    from paper_2104_01253_gb300 import partitioned as pt
    import synth
    Ah = synth.config2_operator(args.N)
    r0 = synth.gaussian_vector(Ah.m, 1002)
    n = args.n
    out = {"suite": "part", "m": Ah.m, "n": n, "points": []}
    for P in (1, 2, 4):
        blocks = pt.row_blocks(Ah.m, P)
        ranks = []
        for lo, hi in blocks:
            rp, ci, va, glo, ghi = pt.local_rows(Ah.row_ptr, Ah.col_idx, Ah.val, lo, hi)
            ctx = kc.Context(0)
            ranks.append((ctx, kc.DeviceCSR(synth.CSR(hi - lo, rp, ci, va)),
                          kc.ArnoldiState(hi - lo, n + 1, kc.KC_F64), lo, hi, glo, ghi))

        def expansion():
            for ctx, A_l, st, lo, hi, _, _ in ranks:
                kc.dcgs2_arnoldi_init(ctx, A_l, st, torch.as_tensor(r0[lo:hi], device="cuda"))
            for k in range(n):
                parts = []
                for ctx, A_l, st, lo, hi, glo, ghi in ranks:
                    pieces = [ranks[q][2].w[max(a, glo) - a:min(b, ghi) - a]
                              for q, (a, b) in enumerate(blocks) if max(a, glo) < min(b, ghi)]
                    part = torch.empty(2 * k + 2, dtype=torch.float64, device="cuda")
                    kc.dcgs2_part_reduce(ctx, A_l, st, torch.cat(pieces), part)
                    parts.append(part)
                tot = torch.stack(parts).sum(0)
                for ctx, A_l, st, _, _, _, _ in ranks:
                    kc.dcgs2_part_update(ctx, A_l, st, tot)

        expansion()
        torch.cuda.synchronize()
        for r in ranks:
            r[0].timing_enable(True)
        expansion()
        torch.cuda.synchronize()
        per_rank = []
        for r in ranks:
            t = r[0].timing_read()
            r[0].timing_enable(False)
            per_rank.append(sum(v[0] for v in t.values()))
        status = [r[0].read_status() for r in ranks]
        out["points"].append({"P": P, "rows_per_rank": [hi - lo for lo, hi in blocks],
                              "kernel_ms_per_rank": per_rank,
                              "kernel_ms_max": max(per_rank),
                              "steps_per_s_without_communication": n / (max(per_rank) / 1e3),
                              "status": status})
        del ranks
        torch.cuda.synchronize()
    ctx = kc.Context(0)
    A = kc.DeviceCSR(Ah)
    st = kc.ArnoldiState(Ah.m, n + 1, kc.KC_F64)
    rd = torch.as_tensor(r0, device="cuda")
    for timed in (False, True):
        ctx.timing_enable(timed)
        kc.dcgs2_arnoldi_init(ctx, A, st, rd)
        for _ in range(n):
            kc.dcgs2_arnoldi_step(ctx, A, st)
        torch.cuda.synchronize()
    t = ctx.timing_read()
    ctx.timing_enable(False)
    out["unpartitioned_kernel_ms"] = sum(v[0] for v in t.values())
    print(json.dumps(out), flush=True)


def suite_cnn(args):
    """kc_cnn_forward and kc_cnn_train_step (regression loss, no Adam update) on a seeded
    random batch of N x N images with He-initialised weights, after two warm-up calls of
    each: mean time per call (CUDA events) and the forward pass's FLOP rate."""
    import torch
    import paper_2104_01253_gb300 as kc
    from paper_2104_01253_gb300.train import he_init
    ctx = kc.Context(0)
    ctx.set_conv_kernel(args.conv)
    B, N = args.batch, args.N
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

    out = {"suite": "cnn", "N": N, "batch": B, "conv": ["mma.sync", "tcgen05"][args.conv]}
    if args.forward > 0:
        ms = timed(lambda: kc.kc_cnn_forward(ctx, w, x, y, B, N, N), args.forward)
        flop = B * N * N * (4 * 32 * 32 * 9 * 2 + 2 * 32 * 9 * 2)
        out.update(forward_ms=ms, forward_tflops=flop / ms / 1e9)
    if args.train > 0:
        wt = w.clone()
        out["train_step_ms"] = timed(
            lambda: kc.kc_cnn_train_step(ctx, wt, None, None, 0, 0.0, x, e, B, N, N, y),
            args.train)
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.suite:
        if args.suite == "cnn" and args.N == 252:
            args.N = 1024
        return {"steps": suite_steps, "solver": suite_solver, "cnn": suite_cnn,
                "learn": suite_learn, "part": suite_part}[args.suite](args)
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    import paper_2104_01253_gb300 as kc

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    Ah = config2_operator(args.N)
    m, nnz = Ah.m, Ah.nnz
    r0_host = gaussian_vector(m, 1002)
    ctx = kc.Context(local)
    ctx.set_fp64_mode(args.fp64_mode)
    if args.staged is not None:
        ctx.set_staged(args.staged)
    A = kc.DeviceCSR(Ah)
    n = args.n
    st = kc.ArnoldiState(m, n + 1, kc.KC_F64)
    r0 = torch.as_tensor(r0_host, device="cuda")
    stream = torch.cuda.current_stream()

    def expansion_on(op, src):
        kc.dcgs2_arnoldi_init(ctx, op, st, src)
        for _ in range(n):
            kc.dcgs2_arnoldi_step(ctx, op, st)
        kc.dcgs2_arnoldi_finish(ctx, op, st)

    def expansion(src):
        expansion_on(A, src)

    for _ in range(args.warmup):
        expansion(r0)
    torch.cuda.synchronize()
    status = ctx.read_status()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    launches0 = ctx.launch_count()
    ctx.timing_enable(True)
    barrier()
    sampler.start()
    time.sleep(0.2)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        expansion(r0)
    e1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms_total = e0.elapsed_time(e1)
    kern = ctx.timing_read()
    ctx.timing_enable(False)
    launches = ctx.launch_count() - launches0
    ms_total = max_over_ranks(ms_total, ws)
    ms_per = ms_total / args.steps
    value = replica_rate(ws, n, args.steps, ms_total)
    total_bytes, per_kernel_bytes = algorithmic_bytes(m, nnz, n)
    hbm_peak, peak_kind = peaks()
    gbs = total_bytes / (ms_per / 1e3) / 1e9
    # the timed expansions' result, kept for the oracle comparison at the end: H and 4096
    # sampled rows of Q
    H_timed = st.H(n + 1, n).cpu().numpy()
    q_rows = np.sort(np.random.default_rng(7).choice(m, size=min(4096, m), replace=False))
    Q_timed = st.Qbuf[:n + 1, torch.as_tensor(q_rows, device="cuda")].cpu().numpy().T

    # quality of the last expansion: loss of orthogonality and Arnoldi relation
    loo = rre = None
    if not args.no_check:
        loo, rre = quality(kc, ctx, A, st, m, n)

    # per-kernel rooflines over the timed expansions.  FP64 FMAs that run on the FP64 pipe
    # per basis element: 2 in the all-FP64 mode, 1 with offload (S and Q C move to the
    # FP32/INT pipes; the method itself still does 2 per element in each pass).  The FP64
    # peak is derived from unit counts and the clock; the HBM peak is measured.
    per = kernel_rooflines(kern, m, nnz, n, args.steps, ctx.fp64_mode, hbm_peak)
    dom = "reduce"
    d = per[dom]
    f_alu, f_hbm = d["fp64_frac"], d["hbm_frac"]
    if f_hbm >= f_alu:
        roofline = {"bound": "hbm", "achieved": d["hbm_gbs"], "peak": hbm_peak, "unit": "GB/s",
                    "frac": f_hbm, "peak_kind": peak_kind}
    else:
        roofline = {"bound": "alu", "achieved": d["fp64_tflops"], "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": f_alu,
                    "peak_kind": "derived FP64 FMA peak (152 SMs x 2 DFMA/clk x 2.07 GHz), "
                                 "not measured"}
    traffic = None
    if ctx.fp64_mode == 1 and not args.staged and dom in TRAFFIC_RATIO:
        traffic = TRAFFIC_RATIO[dom] * d["bytes_per_launch"]
    roofline.update({"kernel": "fused DCGS2 reduction (the 50 steps' launches; the CGS2 "
                               "finish's two reductions are timed apart)",
                     "traffic": traffic,
                     "traffic_note": "bytes per launch: the ncu DRAM/algorithmic ratio at "
                                     "m = 4.1 M times this run's algorithmic bytes per launch",
                     "avg_launch_ms": d["avg_launch_ms"],
                     "fp64_pipe_tflops": d["fp64_tflops"], "fp64_pipe_frac": f_alu,
                     "method_tflops": d["method_tflops"],
                     "hbm_gbs": d["hbm_gbs"], "hbm_frac": f_hbm,
                     "fp64_fma_on_fp64_pipe_per_basis_element": d["fp64_fma_per_elem"]})

    # the same workload on the same GPU: DCGS2 with every product in FP64, CGS2, MGS
    baselines = {}
    if not args.no_baselines:
        def timed(fn, reps=1):
            fn()
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(reps):
                fn()
            t1.record(stream)
            torch.cuda.synchronize()
            return n * reps / (t0.elapsed_time(t1) / 1e3)
        mode = ctx.fp64_mode
        ctx.set_fp64_mode(0)
        baselines["dcgs2_all_fp64_steps_per_s"] = timed(lambda: expansion(r0), 2)
        ctx.set_fp64_mode(mode)

        def classic(step):
            kc.cgs2_arnoldi_init(ctx, A, st, r0)
            for _ in range(n):
                step(ctx, A, st)
        baselines["cgs2_steps_per_s"] = timed(lambda: classic(kc.cgs2_arnoldi_step))
        baselines["mgs_steps_per_s"] = timed(lambda: classic(kc.mgs_arnoldi_step))
        baselines["note"] = ("same m, n and GPU; CGS2 = Algorithm 3 (3 reductions/step), "
                             "MGS level 1 (one reduction per inner product)")

    # the same expansions on the matrix-free stencil form of the operator (same matrix, bit
    # for bit): the basis generation reads w and writes v (16 bytes a row) instead of the
    # CSR arrays; 7 FP64 FMAs a row keep the stencil kernel on the FP64 pipe
    matrix_free = None
    if not args.no_stencil:
        As = kc.DeviceStencil7(config2_stencil(args.N))
        reps = max(args.steps, 2)
        expansion_on(As, r0)
        torch.cuda.synchronize()
        ctx.timing_enable(True)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            expansion_on(As, r0)
        t1.record(stream)
        torch.cuda.synchronize()
        ks = ctx.timing_read()
        ctx.timing_enable(False)
        ms_sp, cnt_sp = ks.get("spmv", (0.0, 0))
        per_launch = ms_sp / max(cnt_sp, 1)
        gbs_sp = 16 * m / (per_launch / 1e3) / 1e9
        tf_sp = 18 * m / (per_launch / 1e3) / 1e12      # 7 products, beta and s per row
        matrix_free = {
            "operator": "7-point stencil %d^3, coefficients of the CSR matrix (no matrix in "
                        "HBM)" % args.N,
            "dcgs2_steps_per_s": n * reps / (t0.elapsed_time(t1) / 1e3),
            "stencil_kernel": {"avg_launch_ms": per_launch, "launches": cnt_sp,
                               "hbm_gbs": gbs_sp, "hbm_frac": gbs_sp / hbm_peak,
                               "fp64_tflops": tf_sp, "fp64_frac": tf_sp / FP64_PEAK_TFLOPS,
                               "algorithmic_bytes_per_launch": 16 * m,
                               "fp64_flop_per_launch": 18 * m},
            "csr_spmv_avg_launch_ms": kern["spmv"][0] / max(kern["spmv"][1], 1),
        }
        if not args.no_solvers:
            b4 = torch.as_tensor(gaussian_vector(m, 1004), device="cuda")
            As32 = kc.DeviceStencil7(config2_stencil(args.N), dtype=torch.float32)
            for name, prec in (("config4_fp64_gmres50", 0), ("config4_ir_fp32_gmres50", 1)):
                x4 = torch.zeros_like(b4)
                t0.record(stream)
                info = kc.gmres_solve(ctx, As, b4, x4, restart=50, rtol=1e-10, precision=prec,
                                      A32=As32, inner_rtol=1e-4, inner_max_cycles=3)
                t1.record(stream)
                torch.cuda.synchronize()
                info["seconds"] = t0.elapsed_time(t1) / 1e3
                matrix_free[name] = info
            del b4, x4

    # end to end through the C ABI with host buffers: H2D of r0, expansion, D2H of H
    e2e = None
    if not args.no_e2e:
        r0_pin = torch.from_numpy(r0_host).pin_memory()
        r0_dev = torch.empty(m, dtype=torch.float64, device="cuda")
        H_host = torch.empty((n, n + 1), dtype=torch.float64).pin_memory()
        barrier()
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for _ in range(args.steps):
            r0_dev.copy_(r0_pin, non_blocking=True)
            expansion(r0_dev)
            H_host.copy_(st.Hbuf[:n, :n + 1], non_blocking=True)
        e3.record(stream)
        barrier()
        ms_e2e = max_over_ranks(e2.elapsed_time(e3), ws)
        e2e = {"value": replica_rate(ws, n, args.steps, ms_e2e), "unit": "steps/s",
               "h2d_bytes_per_step": m * 8, "d2h_bytes_per_step": n * (n + 1) * 8}

    solvers = None
    if not args.no_solvers:
        solvers = solver_suite(kc, ctx, A, m, stream)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, dt, m_s = cpu_oracle_sample(n)
        cpu = {"value": rate * m_s / m, "unit": "steps/s", "cores": blas_threads(),
               "kind": "oracle",
               "sample": "one %d-step FP64 DCGS2 expansion by the numpy/scipy oracle on the "
                         "same operator family at %d rows (%.1f s), rate scaled by rows to "
                         "m = %d" % (n, m_s, dt, m)}

    parity = None
    if rank == 0 and not args.no_parity:
        parity = full_size_parity(Ah, r0_host, n, H_timed, q_rows, Q_timed)
    del Ah

    if rank == 0:
        line = {
            "metric": "arnoldi_steps_per_s", "value": value, "unit": "steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "dcgs2_arnoldi m=%d n=%d (3D convection-diffusion %d^3, "
                                   "upwind, Pe 50, wind (1,0.5,0.25))" % (m, n, args.N),
                       "nnz": nnz, "step": "one %d-column expansion (init, %d DCGS2 steps, "
                                           "CGS2 finish)" % (n, n),
                       "l2": "inputs larger than L2 (basis %.1f GB)" % (8 * m * (n + 1) / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "hbm_gbs": gbs, "hbm_frac_of_%s" % peak_kind: gbs / hbm_peak,
            "algorithmic_bytes_per_step": total_bytes,
            "loo": loo, "rre": rre, "device_status": status,
            "kernels_ms_per_step": {k: v[0] / args.steps for k, v in kern.items()},
            "kernel_rooflines": per,
            "fp64_mode": ["all-fp64", "fp64-with-float-float-offload",
                          "fp64-exact-digit-reduction-on-tensor-cores"][ctx.fp64_mode],
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "same_gpu_baselines": baselines,
            "gpu_launches": launches, "clocks": clocks,
            "gmres_time_to_1e-10": solvers, "matrix_free": matrix_free,
            "parity_vs_oracle": parity,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
