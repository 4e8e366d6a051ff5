"""Gram-Schmidt Arnoldi-QR variants in plain FP64 numpy (test infrastructure only).

Index convention (0-based): after ``k`` DCGS2 steps, columns q_0 .. q_{k-1} of Q are final,
``w`` is the pending (projected once, unnormalised) vector, and Hessenberg columns
0 .. k-2 are final.  H[i, j] is the coefficient of q_i in A q_j, so A Q_n = Q_{n+1} H.
The paper's 1-based index j maps to k = j - 1.

Pins (tests/test_oracle_arnoldi.py): Arnoldi relation and loss of orthogonality at O(eps),
agreement of DCGS2, CGS2 and MGS Hessenbergs on well-conditioned problems, agreement with
Householder QR (LAPACK) of the Krylov matrix, the k = 0 start, breakdown on A = I, the
diagonal-matrix Lanczos case, and the Manteuffel spectrum through Krylov-Schur.
The QR variants (tests/test_oracle_stability.py): the loss-of-orthogonality classes of
Table 3 over graded condition numbers (CGS eps kappa^2, MGS eps kappa, CGS2 and DCGS2 at
O(eps)), the representation error at O(eps), agreement with Householder QR.  ICWY-MGS
(Section 5): the MGS class eps kappa of Table 3's level-2 MGS row, equality with MGS level 1
in exact arithmetic (agreement on well-conditioned inputs), an exact Arnoldi relation, and
planted mistakes (no L correction, L transposed) that leave its class.
"""
from __future__ import annotations

import numpy as np


def _matvec(A, x):
    return A @ x


class DCGS2Arnoldi:
    """DCGS2-Arnoldi (Algorithm 4, Section 4) with one global reduction per step.

    init(r0): w = r0 unnormalised (the factorised matrix is B = [r0, A Q], Section 1).
    step():   one matvec on the pending w, one fused reduction, the delayed normalisation
              (Pythagorean trick), Stephen's trick for T_k (eq. 30), the projection and
              the lagged representation update (the new subdiagonal entry is set before
              the K column that reads it, H_{j-1,j-2}; eq. 52 shows the term belongs).
    finish(): the last column by CGS2 with an explicit norm (end of Section 3: the n-th
              iteration applies CGS2 with two additional reductions).
    """

    def __init__(self, A, r0, ncap: int):
        self.A = A
        m = r0.shape[0]
        self.m = m
        self.ncap = ncap
        self.Q = np.zeros((m, ncap))
        self.H = np.zeros((ncap, ncap - 1))
        self.K = np.zeros((ncap, ncap - 1))   # K[:, j]: partial column j of H, completed one step late
        self.w = np.array(r0, dtype=np.float64, copy=True)
        self.k = 0
        self.alphas = []
        self.finished = False
        self.breakdown = False

    def step(self):
        k = self.k
        if k + 1 >= self.ncap:
            raise ValueError("basis capacity exhausted")
        Qk = self.Q[:, :k]
        w = self.w
        v = _matvec(self.A, w)                      # v = A w_{j-1} (Section 4, matvec on w)
        # the single global reduction [Q_{1:j-2}, w_{j-1}]^T [w_{j-1}, A w_{j-1}] (Algorithm 4)
        C = Qk.T @ w                                # C_{1:j-2,j-1}
        S = Qk.T @ v                                # S_{1:j-2,j}
        beta = w @ w                                # beta_{j-1}
        s = w @ v                                   # S_{j-1,j}
        alpha2 = beta - C @ C                       # Pythagoras (Algorithm 4)
        if not alpha2 > 0.0:
            raise FloatingPointError("Pythagorean norm is not positive")
        alpha = np.sqrt(alpha2)
        if k >= 1:                                  # H column k-1: K + C, subdiagonal alpha
            self.H[:k, k - 1] = self.K[:k, k - 1] + C
            self.H[k, k - 1] = alpha
            # happy breakdown: A q_{k-1} (nearly) lies in span(Q_k)
            if alpha <= 1e-13 * np.linalg.norm(self.H[:k + 1, k - 1]):
                self.breakdown = True
        T = np.empty(k + 1)
        T[:k] = S / alpha                           # first-projection coefficients
        T[k] = (s - C @ S) / alpha ** 2             # Stephen's trick (eq. 30)
        q = (w - Qk @ C) / alpha                    # reorthogonalise and normalise
        self.Q[:, k] = q
        self.w = v / alpha - Qk @ T[:k] - q * T[k]  # projection
        # K_{1:j-1,j-1} = T - (1/alpha) H_{1:j-1,1:j-2} C (Algorithm 4)
        self.K[:k + 1, k] = T - (self.H[:k + 1, :k] @ C) / alpha
        self.alphas.append(alpha)
        self.k = k + 1
        return alpha

    def finish(self):
        """CGS2 on the pending w: finalises H column k-1 and q_k."""
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
        self.Q[:, k] = u / alpha
        self.finished = True
        return alpha

    def result(self):
        k = self.k
        return self.Q[:, :k + 1].copy(), self.H[:k + 1, :k].copy()


def dcgs2_arnoldi(A, r0, n: int):
    """n DCGS2 steps plus the CGS2 finish: Q (m x (n+1)), H ((n+1) x n)."""
    st = DCGS2Arnoldi(A, r0, n + 1)
    for _ in range(n):
        st.step()
    st.finish()
    return st.result()


def cgs2_arnoldi(A, r0, n: int):
    """CGS2-Arnoldi (Algorithm 3): two projections and a normalisation, 3 reductions/step.

    q_0 = r0/||r0||; column j of H holds S + C above the diagonal and alpha below it
    (H[i, j] = coefficient of q_i in A q_j, eq. "arnoldi").
    """
    m = r0.shape[0]
    Q = np.zeros((m, n + 1))
    H = np.zeros((n + 1, n))
    Q[:, 0] = r0 / np.sqrt(r0 @ r0)
    for j in range(n):
        Qj = Q[:, :j + 1]
        v = _matvec(A, Q[:, j])                     # generation of the next vector
        S = Qj.T @ v                                # first projection
        w = v - Qj @ S
        C = Qj.T @ w                                # second projection
        u = w - Qj @ C
        alpha = np.sqrt(u @ u)                      # normalisation
        Q[:, j + 1] = u / alpha
        H[:j + 1, j] = S + C
        H[j + 1, j] = alpha
    return Q, H


def mgs_arnoldi(A, r0, n: int):
    """MGS-Arnoldi, level 1: sequential rank-1 projections, one reduction per inner product."""
    m = r0.shape[0]
    Q = np.zeros((m, n + 1))
    H = np.zeros((n + 1, n))
    Q[:, 0] = r0 / np.sqrt(r0 @ r0)
    for j in range(n):
        v = _matvec(A, Q[:, j])
        for i in range(j + 1):
            h = Q[:, i] @ v
            v = v - h * Q[:, i]
            H[i, j] = h
        alpha = np.sqrt(v @ v)
        H[j + 1, j] = alpha
        Q[:, j + 1] = v / alpha
    return Q, H


def cgs_qr(B):
    """Classical Gram-Schmidt QR, one projection pass (Algorithm 1 without its second
    projection): the O(eps) kappa^2 loss-of-orthogonality class of Table 3."""
    m, n = B.shape
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    for j in range(n):
        a = B[:, j]
        S = Q[:, :j].T @ a
        u = a - Q[:, :j] @ S
        alpha = np.sqrt(u @ u)
        Q[:, j] = u / alpha
        R[:j, j] = S
        R[j, j] = alpha
    return Q, R


def mgs_qr(B):
    """Modified Gram-Schmidt QR, level 1 (Section 2: the rank-1 projections I - q_i q_i^T
    applied one after another, one inner product each): the O(eps) kappa class of Table 3."""
    m, n = B.shape
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    for j in range(n):
        u = np.array(B[:, j], dtype=np.float64)
        for i in range(j):
            R[i, j] = Q[:, i] @ u
            u = u - R[i, j] * Q[:, i]
        R[j, j] = np.sqrt(u @ u)
        Q[:, j] = u / R[j, j]
    return Q, R


def cgs2_qr(B):
    """CGS2 QR of B (Algorithm 1): B = Q R, R upper triangular with R_jj = alpha_j."""
    m, n = B.shape
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    for j in range(n):
        a = B[:, j]
        Qj = Q[:, :j]
        S = Qj.T @ a
        w = a - Qj @ S
        C = Qj.T @ w
        u = w - Qj @ C
        alpha = np.sqrt(u @ u)
        Q[:, j] = u / alpha
        R[:j, j] = S + C
        R[j, j] = alpha
    return Q, R


def dcgs2_qr(B):
    """DCGS2 QR of B (Algorithm 2): one reduction per column, last column by CGS2.

    At iteration j (0-based, j >= 1) the reduction [Q_{0:j-2}, w_{j-1}]^T [w_{j-1}, a_j]
    gives C (delayed reorthogonalisation of w_{j-1}), beta, S_{0:j-2} and S_{j-1}; then
    alpha_{j-1} by Pythagoras, q_{j-1}, Stephen's trick for S_{j-1,j}, the projection of
    a_j, and column j-1 of R (S of the previous iteration plus C).
    """
    m, n = B.shape
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    w = B[:, 0].copy()                 # w_0 = a_0 (nothing to project against)
    S_prev = np.zeros(0)               # S_{0:j-2, j-1} of the previous iteration
    for j in range(1, n):
        a = B[:, j]
        Qp = Q[:, :j - 1]              # Q_{0:j-2}
        C = Qp.T @ w
        beta = w @ w
        S = Qp.T @ a
        s = w @ a
        alpha = np.sqrt(beta - C @ C)
        q = (w - Qp @ C) / alpha
        Q[:, j - 1] = q
        s_corr = (s - C @ S) / alpha   # Stephen's trick: q_{j-1}^T a_j
        R[:j - 1, j - 1] = S_prev + C
        R[j - 1, j - 1] = alpha
        S_full = np.concatenate([S, [s_corr]])
        w = a - Q[:, :j] @ S_full
        S_prev = S_full
    # last column: CGS2 with explicit norm
    Qp = Q[:, :n - 1]
    C1 = Qp.T @ w
    u = w - Qp @ C1
    C2 = Qp.T @ u
    u = u - Qp @ C2
    alpha = np.sqrt(u @ u)
    Q[:, n - 1] = u / alpha
    R[:n - 1, n - 1] = S_prev + C1 + C2
    R[n - 1, n - 1] = alpha
    return Q, R


def _forward_solve_unit_lower(L, r):
    """y with (I + L) y = r, L strictly lower triangular (forward substitution)."""
    y = np.array(r, dtype=np.float64, copy=True)
    for i in range(y.shape[0]):
        y[i] -= L[i, :i] @ y[:i]
    return y


def icwy_qr(B):
    """ICWY-MGS QR of B (Section 5): the inverse compact WY projector
    P a = (I - Q T Q^T) a with T = (I + L)^{-1}, L strictly lower triangular whose row i
    holds the inner products q_i^T q_{0:i-1} (the strictly lower part of Q^T Q).  One
    reduction per column: at iteration j (j >= 1) the single reduction
    [Q_{0:j-2}, u_{j-1}]^T [u_{j-1}, a_j] gives row j-1 of L (scaled by the norm), the
    norm of the pending u_{j-1} and Q^T a_j; then q_{j-1} = u_{j-1} / ||u_{j-1}||,
    R(0:j, j) = (I + L)^{-1} Q_{0:j-1}^T a_j and u_j = a_j - Q_{0:j-1} R(0:j, j).  The last
    column is normalised by one more reduction."""
    m, n = B.shape
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    L = np.zeros((n, n))
    u = np.array(B[:, 0], dtype=np.float64, copy=True)       # u_0 = a_0
    for j in range(1, n):
        a = B[:, j]
        Qp = Q[:, :j - 1]
        ell = Qp.T @ u                    # the one reduction: Q^T u, u^T u, Q^T a, u^T a
        beta = u @ u
        r = Qp.T @ a
        rho = u @ a
        alpha = np.sqrt(beta)
        Q[:, j - 1] = u / alpha
        R[j - 1, j - 1] = alpha
        L[j - 1, :j - 1] = ell / alpha    # row j-1 of L: q_{j-1}^T q_{0:j-2}
        y = _forward_solve_unit_lower(L[:j, :j], np.concatenate([r, [rho / alpha]]))
        R[:j, j] = y
        u = a - Q[:, :j] @ y
    alpha = np.sqrt(u @ u)
    Q[:, n - 1] = u / alpha
    R[n - 1, n - 1] = alpha
    return Q, R


def icwy_arnoldi(A, r0, n: int):
    """ICWY-MGS Arnoldi (Section 5's projector in the Arnoldi expansion, one reduction per
    step).  The pending vector w is the projected, unnormalised A q_{k-1} (w = r0 at the
    start); step k applies A to w (v = A w, so A q_k = v / alpha), and its one reduction
    [Q_k, w]^T [w, v] gives C = Q_k^T w, S = Q_k^T v, beta = w^T w and s = w^T v.  Then
    alpha = sqrt(beta), q_k = w / alpha, H(k, k-1) = alpha, row k of L = C / alpha,
    H(0:k+1, k) = (I + L)^{-1} [S / alpha; s / alpha^2] and w <- v / alpha - Q_{k+1} H(0:k+1, k).
    The last column is normalised by one more reduction.  Q (m x (n+1)), H ((n+1) x n)."""
    m = r0.shape[0]
    Q = np.zeros((m, n + 1))
    H = np.zeros((n + 1, n))
    L = np.zeros((n + 1, n + 1))
    w = np.array(r0, dtype=np.float64, copy=True)
    for k in range(n):
        v = _matvec(A, w)
        Qk = Q[:, :k]
        C = Qk.T @ w                      # the one reduction of the step
        S = Qk.T @ v
        beta = w @ w
        s = w @ v
        alpha = np.sqrt(beta)
        Q[:, k] = w / alpha
        if k >= 1:
            H[k, k - 1] = alpha
        L[k, :k] = C / alpha
        y = _forward_solve_unit_lower(L[:k + 1, :k + 1],
                                      np.concatenate([S / alpha, [s / alpha ** 2]]))
        H[:k + 1, k] = y
        w = v / alpha - Q[:, :k + 1] @ y
    alpha = np.sqrt(w @ w)
    H[n, n - 1] = alpha
    Q[:, n] = w / alpha
    return Q, H
