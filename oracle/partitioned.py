"""Row-partitioned DCGS2 Arnoldi (Algorithm 4) over P ranks, the paper's distributed
layout (Section 5: Q, w, v and the rows of A split by rows across processes, one global
reduction per step), written as an oracle so that the partition can be checked on CPU
ranks (torch.distributed with the gloo backend) against the sequential oracle.

Per step k, rank p holds rows [r_p, r_{p+1}) of A, Q, w and v.  It gathers w (standing in
for the halo exchange of a stencil SpMV), forms its rows of v = A w, computes its partial
[Q_k, w]^T [w, v] (C, S, beta, s: 2k + 2 numbers) and takes part in ONE all-reduce (sum)
of them; the scalar step (Pythagoras, Stephen's trick, the H and K columns) is replicated,
and the update of q_k and w is row-local.  The CGS2 finish needs three more all-reduces
(two projections and the norm).

Test infrastructure, like the rest of this package: only the tests use it.
Pins: tests/test_partitioned_oracle.py (agreement with oracle.arnoldi.dcgs2_arnoldi on
2 and 3 ranks, and the count of all-reduces per step).
"""
from __future__ import annotations

import numpy as np


def row_blocks(m: int, P: int):
    """Contiguous row ranges of P ranks, sizes differing by at most one."""
    b = [(m * p) // P for p in range(P + 1)]
    return list(zip(b[:-1], b[1:]))


def dcgs2_arnoldi_rows(A, r0, n, rank, P, allreduce_sum, allgather):
    """DCGS2 Arnoldi on this rank's rows.  A: scipy CSR (all rows; the rank reads only its
    own), r0: full start vector (the rank keeps its rows), allreduce_sum(x) returns the
    sum of x over ranks, allgather(x_local) returns the full vector.  Returns this rank's
    rows of Q_{n+1} and the replicated H ((n+1) x n)."""
    lo, hi = row_blocks(A.shape[0], P)[rank]
    Al = A[lo:hi]
    ml = hi - lo
    Q = np.zeros((ml, n + 1))
    H = np.zeros((n + 1, n))
    K = np.zeros((n + 1, n + 1))
    w = np.array(r0[lo:hi], dtype=np.float64)
    for k in range(n):
        v = Al @ allgather(w)                                # rows of v = A w
        Qk = Q[:, :k]
        part = np.concatenate([Qk.T @ w, Qk.T @ v, [w @ w, w @ v]])
        tot = allreduce_sum(part)                            # the one reduction of step k
        C, S, beta, s = tot[:k], tot[k:2 * k], tot[2 * k], tot[2 * k + 1]
        a2 = beta - C @ C                                    # Pythagoras (Algorithm 4)
        if not a2 > 0.0:
            raise FloatingPointError("beta - C^T C <= 0 at step %d" % k)
        alpha = np.sqrt(a2)
        if k >= 1:
            H[:k, k - 1] = K[:k, k - 1] + C                  # H column: K + C
            H[k, k - 1] = alpha                              # subdiagonal
        T = np.concatenate([S / alpha, [(s - C @ S) / alpha ** 2]])   # Stephen's trick, eq. 30
        q = (w - Qk @ C) / alpha                             # reorthogonalise
        Q[:, k] = q
        K[:k + 1, k] = T - H[:k + 1, :k] @ C / alpha         # lagged correction
        w = v / alpha - Qk @ T[:k] - q * T[k]                # projection
    # CGS2 finish of the last column (explicit norm)
    Qn = Q[:, :n]
    C1 = allreduce_sum(Qn.T @ w)
    u = w - Qn @ C1
    C2 = allreduce_sum(Qn.T @ u)
    u = u - Qn @ C2
    alpha = np.sqrt(allreduce_sum(np.array([u @ u]))[0])
    H[:n, n - 1] = K[:n, n - 1] + C1 + C2
    H[n, n - 1] = alpha
    Q[:, n] = u / alpha
    return Q, H
