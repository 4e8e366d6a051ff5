"""Restarted GMRES / FGMRES on DCGS2-Arnoldi, and FP64 iterative refinement (test only).

gmres():  textbook restarted GMRES (Saad and Schultz) whose Arnoldi process is the DCGS2
          step of Algorithm 4.  Hessenberg columns arrive one step late (column k-1 is
          final after step k), so the Givens rotations and the residual estimate |g_k| lag
          one step behind the matvec; the CGS2 finish closes a full cycle.  The paper gives
          no GMRES details beyond using the Arnoldi-QR expansion (Section 1).
fgmres(): flexible right preconditioning.  With a preconditioner M the DCGS2 step works on
          v = A M(w) and stores z_k = M(w_k)/alpha_k; then A z_k = v/alpha_k =
          w_{k+1} + Q_{k+1} T, so column k of H is T + C_{k+1} with no H*C/alpha correction.
ir():     FP64 iterative refinement around an inner GMRES run in float32 arithmetic, the
          basis stored either in float32 or rounded to bfloat16 (round to nearest even).

The arithmetic type of the inner solve is a parameter (numpy float64 or float32).
Pins: tests/test_oracle_gmres.py (scipy spsolve solutions, the true residual of the
returned x, the residual-estimate identity |g_k| = ||b - A x_k||, iterative refinement
reaching 1e-10 with a float32 inner solve, FGMRES with the identity and with a linear
preconditioner against GMRES on the preconditioned system).
"""
from __future__ import annotations

import numpy as np


def round_bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float32."""
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


class _Arnoldi:
    """DCGS2-Arnoldi steps in a chosen float type, optionally flexible (Algorithm 4)."""

    def __init__(self, A, r0, ncap, dtype, q_round=None, precond=None):
        self.A = A
        self.dtype = dtype
        m = r0.shape[0]
        self.Q = np.zeros((m, ncap), dtype=dtype)
        self.Z = np.zeros((m, ncap), dtype=dtype) if precond is not None else None
        self.H = np.zeros((ncap, ncap - 1), dtype=np.float64)
        self.K = np.zeros((ncap, ncap - 1), dtype=dtype)
        self.w = np.asarray(r0, dtype=dtype).copy()
        self.k = 0
        self.q_round = q_round
        self.precond = precond
        self.pyth_fallbacks = 0

    def step(self):
        k = self.k
        dt = self.dtype
        Qk = self.Q[:, :k]
        w = self.w
        if self.precond is None:
            v = (self.A @ w).astype(dt)
        else:
            zhat = np.asarray(self.precond(w), dtype=dt)
            v = (self.A @ zhat).astype(dt)
        C = Qk.T @ w
        S = Qk.T @ v
        beta = w @ w
        s = w @ v
        alpha2 = beta - C @ C
        eps = np.finfo(dt).eps
        if not alpha2 > 64 * eps * beta:
            # Pythagoras lost its digits: explicit norm of u = w - Q C instead
            u = w - Qk @ C
            alpha2 = u @ u
            self.pyth_fallbacks += 1
        alpha = dt(np.sqrt(alpha2))
        if k >= 1:
            self.H[:k, k - 1] = self.K[:k, k - 1] + C
            self.H[k, k - 1] = alpha
        T = np.empty(k + 1, dtype=dt)
        T[:k] = S / alpha
        T[k] = (s - C @ S) / (alpha * alpha)
        q = (w - Qk @ C) / alpha
        if self.q_round is not None:
            q = self.q_round(q)
        self.Q[:, k] = q
        self.w = v / alpha - Qk @ T[:k] - q * T[k]
        if self.precond is None:
            self.K[:k + 1, k] = T - (self.H[:k + 1, :k].astype(dt) @ C) / alpha
        else:
            self.Z[:, k] = zhat / alpha
            self.K[:k + 1, k] = T
        self.k = k + 1
        return float(alpha)

    def finish(self):
        k = self.k
        Qk = self.Q[:, :k]
        w = self.w
        C1 = Qk.T @ w
        u = w - Qk @ C1
        C2 = Qk.T @ u
        u = u - Qk @ C2
        alpha = np.sqrt(u @ u)
        self.H[:k, k - 1] = self.K[:k, k - 1] + C1 + C2
        self.H[k, k - 1] = alpha


class _Givens:
    """Incremental QR of the (k+1) x k Hessenberg matrix by Givens rotations (FP64)."""

    def __init__(self, n, gamma):
        self.R = np.zeros((n + 1, n))
        self.c = np.zeros(n)
        self.s = np.zeros(n)
        self.g = np.zeros(n + 1)
        self.g[0] = gamma
        self.j = 0

    def add_column(self, h):
        j = self.j
        h = np.array(h[:j + 2], dtype=np.float64)
        for i in range(j):
            t = self.c[i] * h[i] + self.s[i] * h[i + 1]
            h[i + 1] = -self.s[i] * h[i] + self.c[i] * h[i + 1]
            h[i] = t
        r = np.hypot(h[j], h[j + 1])
        self.c[j] = h[j] / r
        self.s[j] = h[j + 1] / r
        h[j] = r
        h[j + 1] = 0.0
        self.R[:j + 1, j] = h[:j + 1]
        self.g[j + 1] = -self.s[j] * self.g[j]
        self.g[j] = self.c[j] * self.g[j]
        self.j = j + 1
        return abs(self.g[j + 1])

    def solve(self):
        j = self.j
        y = np.zeros(j)
        for i in range(j - 1, -1, -1):
            y[i] = (self.g[i] - self.R[i, i + 1:j] @ y[i + 1:j]) / self.R[i, i]
        return y


def gmres(A, b, restart=30, rtol=1e-10, maxit=10000, x0=None, dtype=np.float64,
          q_round=None, precond=None, max_restarts=None):
    """Restarted (F)GMRES with DCGS2-Arnoldi.  Returns (x, info).

    Stops when the residual estimate |g_k| / ||b|| <= rtol, or after ``maxit`` matvecs, or
    after ``max_restarts`` cycles.  info: iters (matvecs), restarts, rel_resid_est,
    rel_resid_true (recomputed in FP64), history (per-step estimates).
    """
    dt = dtype
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    A_dt = A.astype(dt) if dt != np.float64 else A
    bnorm = np.linalg.norm(b)
    iters = 0
    restarts = 0
    history = []
    est = np.inf
    while True:
        r = b - A @ x
        gamma = np.linalg.norm(r)
        if gamma / bnorm <= rtol or iters >= maxit:
            est = gamma / bnorm
            break
        if max_restarts is not None and restarts >= max_restarts:
            est = gamma / bnorm
            break
        arn = _Arnoldi(A_dt, r.astype(dt), restart + 1, dt, q_round, precond)
        giv = None
        ncols = 0
        converged = False
        stopped = False
        for step in range(restart):
            alpha = arn.step()
            iters += 1
            if step == 0:
                giv = _Givens(restart, alpha)       # alpha_0 = ||r||
                continue
            est = giv.add_column(arn.H[:, step - 1]) / bnorm
            history.append(est)
            ncols = step
            if est <= rtol:
                converged = True
                break
            if iters >= maxit and step < restart - 1:
                stopped = True
                break
        if not (converged or stopped):
            arn.finish()
            est = giv.add_column(arn.H[:, restart - 1]) / bnorm
            history.append(est)
            ncols = restart
        y = giv.solve()
        basis = arn.Z if precond is not None else arn.Q
        x = x + (basis[:, :ncols].astype(np.float64) @ y)
        restarts += 1
        if converged and est <= rtol:
            r = b - A @ x
            if np.linalg.norm(r) / bnorm <= rtol or iters >= maxit:
                est = np.linalg.norm(r) / bnorm
                break
        if iters >= maxit:
            break
    true = np.linalg.norm(b - A @ x) / bnorm
    return x, dict(iters=iters, restarts=restarts, rel_resid_est=float(est),
                   rel_resid_true=float(true), history=history)


def ir(A, b, restart=50, rtol=1e-10, inner_rtol=1e-4, inner_max_restarts=2,
       basis="f32", max_outer=50):
    """FP64 iterative refinement with an FP32 DCGS2-GMRES inner solve.

    x = 0; repeat: r = b - A x (FP64); stop when ||r||/||b|| <= rtol; solve
    A_32 d = r/||r|| by float32 GMRES(restart) to inner_rtol (at most
    inner_max_restarts + 1 cycles); x += ||r|| d.  basis: "f32" or "bf16" (Q rounded to
    bfloat16 on store, all dot products and updates in float32).
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    q_round = round_bf16 if basis == "bf16" else None
    A32 = A.astype(np.float32)
    outer = 0
    inner_iters = 0
    hist = []
    while True:
        r = b - A @ x
        rn = np.linalg.norm(r)
        hist.append(rn / bnorm)
        if rn / bnorm <= rtol or outer >= max_outer:
            break
        d, info = gmres(A32, (r / rn).astype(np.float32), restart=restart, rtol=inner_rtol,
                        dtype=np.float32, q_round=q_round,
                        max_restarts=inner_max_restarts + 1)
        inner_iters += info["iters"]
        x = x + rn * d
        outer += 1
    return x, dict(outer=outer, inner_iters=inner_iters, rel_resid_true=float(hist[-1]),
                   history=hist)
