"""Krylov-Schur eigenvalues on DCGS2-Arnoldi (test infrastructure only).

Stewart's Krylov-Schur restart (cited in Section 1; used for the Manteuffel experiments of
Section 6.1): expand a Krylov decomposition A Q_n = Q_n B + q_n b^T to n = ncv columns with
DCGS2 steps, take the real Schur form B = Z T Z^T ordered so that the wanted Ritz values
(largest real part) lead, test each wanted Ritz pair by its Arnoldi residual
||(A - lambda I) Q Z y|| = |b^T Z y| (eq. "ArnoldiRes"), keep p columns
(p = nkeep, or nkeep + 1 if a complex pair would be split), and restart from
Q_p <- Q_n Z[:, :p], q_p <- q_n, B <- T[:p, :p], b <- Z[:, :p]^T b.

After a truncation the new expansion starts with a single projection of A q_p (the first
half of CGS2, whose second half is the next DCGS2 step's delayed reorthogonalisation);
the DCGS2 correction K = T - H C / alpha uses full H rows, so it stays valid for the
non-Hessenberg leading block.  The small dense Schur step is LAPACK (scipy.linalg.schur),
a library primitive.

Pins: tests/test_oracle_ks.py (dense eigenvalues of small operators, the Manteuffel closed
form, the Arnoldi residual identity).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def wanted_set(evals, p):
    """Indices of the p eigenvalues of largest real part (ties: larger imag, then index),
    widened to p+1 when the p-th and (p+1)-th form a complex-conjugate pair."""
    order = sorted(range(len(evals)), key=lambda i: (-evals[i].real, -evals[i].imag, i))
    sel = order[:p]
    last = evals[order[p - 1]]
    if p < len(order) and abs(last.imag) > 0.0:
        partner = np.conj(last)
        if not any(abs(evals[i] - partner) <= 1e-14 * max(1.0, abs(partner)) for i in sel):
            sel = order[:p + 1]
    return sel


class KrylovSchur:
    def __init__(self, A, v0, nev=10, ncv=40, nkeep=20, tol=1e-10):
        self.A = A
        self.nev, self.ncv, self.nkeep, self.tol = nev, ncv, nkeep, tol
        m = v0.shape[0]
        self.Q = np.zeros((m, ncv + 1))
        self.H = np.zeros((ncv + 1, ncv))
        self.K = np.zeros((ncv + 1, ncv))
        self.w = np.array(v0, dtype=np.float64)
        self.k = 0
        self.matvecs = 0

    # --- DCGS2 expansion (Algorithm 4) ---------------------------------------------------
    def _dcgs2_step(self):
        k = self.k
        Qk = self.Q[:, :k]
        w = self.w
        v = self.A @ w
        self.matvecs += 1
        C = Qk.T @ w
        S = Qk.T @ v
        beta = w @ w
        s = w @ v
        alpha = np.sqrt(beta - C @ C)
        if k >= 1:
            self.H[:k, k - 1] = self.K[:k, k - 1] + C
            self.H[k, k - 1] = alpha
        T = np.empty(k + 1)
        T[:k] = S / alpha
        T[k] = (s - C @ S) / alpha ** 2
        q = (w - Qk @ C) / alpha
        self.Q[:, k] = q
        self.w = v / alpha - Qk @ T[:k] - q * T[k]
        self.K[:k + 1, k] = T - (self.H[:k + 1, :k] @ C) / alpha
        self.k = k + 1

    def _finish(self):
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

    def _project_restart(self, p):
        """Pending vector after truncation: one projection of A q_p onto Q_{p+1}."""
        Qp = self.Q[:, :p + 1]
        v = self.A @ self.Q[:, p]
        self.matvecs += 1
        S = Qp.T @ v
        self.w = v - Qp @ S
        self.K[:, p] = 0.0
        self.K[:p + 1, p] = S
        self.k = p + 1

    def expand(self):
        while self.k < self.ncv:
            self._dcgs2_step()
        self._finish()

    # --- Schur step, convergence test, truncation ----------------------------------------
    def schur_step(self):
        n = self.ncv
        B = self.H[:n, :n]
        b = self.H[n, :n]
        evals = np.linalg.eigvals(B)
        p = len(wanted_set(evals, self.nkeep))
        sel_vals = [evals[i] for i in wanted_set(evals, self.nkeep)]

        def sortf(re, im):
            z = complex(re, im)
            return any(abs(z - s) <= 1e-12 * max(1.0, abs(s)) for s in sel_vals)

        T, Z, sdim = sla.schur(B, output="real", sort=sortf)
        if sdim != p:
            raise RuntimeError("Schur reordering selected %d of %d values" % (sdim, p))
        # Ritz values of the leading block and their Arnoldi residuals
        lam, Y = sla.eig(T[:p, :p])
        bt = b @ Z[:, :p]
        res = np.abs(bt @ Y) / np.linalg.norm(Y, axis=0)
        order = sorted(range(p), key=lambda i: (-lam[i].real, -lam[i].imag, i))
        lam = lam[order]
        res = res[order]
        return T, Z, p, lam, res

    def truncate(self, T, Z, p):
        n = self.ncv
        b = self.H[n, :n].copy()
        Qn = self.Q[:, :n].copy()
        self.Q[:, :p] = Qn @ Z[:, :p]
        self.Q[:, p] = self.Q[:, n]
        self.H[:] = 0.0
        self.H[:p, :p] = T[:p, :p]
        self.H[p, :p] = b @ Z[:, :p]
        self._project_restart(p)

    def run(self, maxrestarts=500):
        self.expand()
        restarts = 0
        while True:
            T, Z, p, lam, res = self.schur_step()
            wanted = lam[:self.nev]
            conv = res[:self.nev] <= self.tol * np.maximum(np.abs(wanted), 1e-300)
            nconv = int(np.sum(conv))
            if nconv >= self.nev or restarts >= maxrestarts:
                return dict(eigs=wanted, resid=res[:self.nev], nconv=nconv,
                            restarts=restarts, matvecs=self.matvecs)
            self.truncate(T, Z, p)
            self.expand()
            restarts += 1


def krylov_schur(A, v0, nev=10, ncv=40, nkeep=20, tol=1e-10, maxrestarts=500):
    return KrylovSchur(A, v0, nev, ncv, nkeep, tol).run(maxrestarts)
