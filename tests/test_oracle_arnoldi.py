"""Pins of the FP64 oracle's Gram-Schmidt Arnoldi-QR variants (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import arnoldi as orc
from oracle.metrics import loo, rre
from synth import convdiff_csr, gaussian_vector, manteuffel_csr


def _random_sparse(m, seed, density=0.05):
    rng = np.random.default_rng(seed)
    A = sp.random(m, m, density=density, random_state=rng, format="csr")
    return (A + 4.0 * sp.eye(m)).tocsr()


@pytest.fixture(scope="module")
def mant():
    return manteuffel_csr(20).to_scipy()


@pytest.mark.parametrize("variant", [orc.dcgs2_arnoldi, orc.cgs2_arnoldi, orc.mgs_arnoldi])
def test_arnoldi_relation(mant, variant):
    """A Q_n = Q_{n+1} H_n to O(eps) (eq. "arnoldi"; RRE of Section 6.1)."""
    r0 = gaussian_vector(mant.shape[0], 1)
    Q, H = variant(mant, r0, 40)
    assert rre(mant, Q, H) < 1e-15
    # H is upper Hessenberg with a positive subdiagonal
    assert np.all(np.tril(H, -2) == 0.0)
    assert np.all(np.diag(H, -1) > 0.0)


@pytest.mark.parametrize("variant,bound", [(orc.dcgs2_arnoldi, 1e-14), (orc.cgs2_arnoldi, 1e-14)])
def test_loss_of_orthogonality_eps(mant, variant, bound):
    """CGS2 and DCGS2 keep ||I - Q^T Q||_F at O(eps) (Table 3)."""
    r0 = gaussian_vector(mant.shape[0], 2)
    Q, H = variant(mant, r0, 60)
    assert loo(Q) < bound


def test_mgs_loses_more_orthogonality_than_dcgs2():
    """MGS loses orthogonality like eps*kappa, DCGS2 stays at eps (Table 3, Section 6.1)."""
    A = manteuffel_csr(30).to_scipy()
    r0 = gaussian_vector(A.shape[0], 3)
    Qm, _ = orc.mgs_arnoldi(A, r0, 80)
    Qd, _ = orc.dcgs2_arnoldi(A, r0, 80)
    assert loo(Qd) < 1e-14
    assert loo(Qm) > 20 * loo(Qd)


def test_dcgs2_equals_cgs2_and_mgs_in_exact_arithmetic():
    """DCGS2, CGS2 and MGS produce the same Q and H (derivation of Section 4) on a
    well-conditioned problem, up to rounding."""
    A = _random_sparse(300, 4)
    r0 = gaussian_vector(300, 4)
    Qd, Hd = orc.dcgs2_arnoldi(A, r0, 20)
    Qc, Hc = orc.cgs2_arnoldi(A, r0, 20)
    Qm, Hm = orc.mgs_arnoldi(A, r0, 20)
    assert np.linalg.norm(Hd - Hc) / np.linalg.norm(Hc) < 1e-13
    # MGS only keeps orthogonality to O(eps * kappa), so its H agrees less tightly
    assert np.linalg.norm(Hd - Hm) / np.linalg.norm(Hm) < 1e-9
    assert np.abs(Qd - Qc).max() < 1e-12


def test_krylov_basis_matches_householder_qr():
    """Q_{n+1} spans K_{n+1}(A, r0): compare with LAPACK Householder QR of the Krylov
    matrix [r0, A r0, ..., A^n r0] (columns agree up to sign)."""
    A = _random_sparse(200, 5)
    r0 = gaussian_vector(200, 5)
    n = 6
    Kry = np.empty((200, n + 1))
    Kry[:, 0] = r0
    for j in range(n):
        Kry[:, j + 1] = A @ Kry[:, j]
    Qh, Rh = np.linalg.qr(Kry)
    Qd, Hd = orc.dcgs2_arnoldi(A, r0, n)
    signs = np.sign(np.diag(Rh))
    assert np.abs(Qd - Qh * signs).max() < 1e-9


def test_first_step_normalises_r0():
    """k = 0: q_0 = r0/||r0|| and alpha_0 = ||r0|| (start of the expansion, B = [r0, AQ])."""
    A = _random_sparse(100, 6)
    r0 = gaussian_vector(100, 6)
    st = orc.DCGS2Arnoldi(A, r0, 5)
    alpha = st.step()
    assert abs(alpha - np.linalg.norm(r0)) < 1e-13 * np.linalg.norm(r0)
    assert np.abs(st.Q[:, 0] - r0 / np.linalg.norm(r0)).max() < 1e-15


def test_identity_breaks_down_at_step_one():
    """A = I: A r0 lies in span{r0}, so the second normalisation has nothing left: either
    Pythagoras gives no positive norm or alpha_1 is at rounding level (happy breakdown)."""
    A = sp.eye(50, format="csr")
    st = orc.DCGS2Arnoldi(A, gaussian_vector(50, 7), 5)
    st.step()
    try:
        st.step()
    except FloatingPointError:
        return
    assert st.breakdown
    assert st.H[1, 0] < 1e-13 * abs(st.H[0, 0])


def test_symmetric_matrix_gives_lanczos_tridiagonal():
    """For symmetric A, Arnoldi reduces to Lanczos: H is symmetric tridiagonal."""
    d = np.linspace(1.0, 3.0, 400)
    A = sp.diags(d).tocsr()
    Q, H = orc.dcgs2_arnoldi(A, np.ones(400), 25)
    Hs = H[:25, :25]
    assert np.abs(np.triu(Hs, 2)).max() < 1e-12
    assert np.abs(Hs - Hs.T).max() < 1e-12
    # first diagonal entry is the Rayleigh quotient mean(d) for r0 = ones
    assert abs(H[0, 0] - d.mean()) < 1e-14


def test_full_arnoldi_ritz_values_are_eigenvalues():
    """With n = m the Ritz values (eigenvalues of H_m) are exactly the eigenvalues of A."""
    A = manteuffel_csr(4).to_scipy()        # m = 16, real spectrum from the closed form
    st = orc.DCGS2Arnoldi(A, gaussian_vector(16, 8), 17)
    for _ in range(16):
        st.step()
    Hs = st.H[:16, :15]
    # columns 0..14 final; last column from the pending w projected (breakdown is exact)
    ev_h = np.sort(np.linalg.eigvals(np.column_stack([Hs[:16], st.K[:16, 15]])).real)
    ev_a = np.sort(np.linalg.eigvals(A.toarray()).real)
    assert np.abs(ev_h - ev_a).max() < 1e-10


@pytest.mark.parametrize("qr", [orc.dcgs2_qr, orc.cgs2_qr])
def test_qr_variants_match_householder(qr):
    """CGS2 (Algorithm 1) and DCGS2 (Algorithm 2) QR equal Householder QR up to signs."""
    B = np.random.default_rng(9).standard_normal((500, 30))
    Q, R = qr(B)
    Qh, Rh = np.linalg.qr(B)
    s = np.sign(np.diag(Rh))
    assert np.abs(R - s[:, None] * Rh).max() < 1e-12
    assert loo(Q) < 1e-14
    assert np.linalg.norm(Q @ R - B) / np.linalg.norm(B) < 1e-15


def test_partitioned_reduction_matches_unpartitioned():
    """Row-partitioned partial sums (the paper's data-parallel layout, m/p rows per rank)
    reproduce the one-reduction quantities to rounding."""
    A = convdiff_csr(12, 3, [1.0, 0.5, 0.25])
    Asp = A.to_scipy()
    r0 = gaussian_vector(A.m, 10)
    st = orc.DCGS2Arnoldi(Asp, r0, 12)
    for _ in range(8):
        st.step()
    Q = st.Q[:, :8]
    w = st.w
    v = Asp @ w
    full = np.concatenate([Q.T @ w, Q.T @ v, [w @ w, w @ v]])
    parts = np.array_split(np.arange(A.m), 4)
    summed = sum(np.concatenate([Q[p].T @ w[p], Q[p].T @ v[p], [w[p] @ w[p], w[p] @ v[p]]])
                 for p in parts)
    assert np.abs(summed - full).max() < 1e-12 * np.abs(full).max()


def _crafted_step_errors(cls):
    """DCGS2 from a crafted state whose delayed coefficients C are O(1), not O(eps).

    A CGS2 run gives Q_5 and H (A Q_4 = Q_5 H).  The DCGS2 state is set to k = 3 with the
    pending vector w = alpha_3 q_3 + Q_3 c (c random, O(1)) and K[:, 2] = H[:3, 2] - c, so
    the delayed reorthogonalisation must remove c.  One step plus the CGS2 finish must
    reproduce alpha_3 (Pythagoras), q_3, column 2 of H, and column 3 of H (which needs
    the correction H C / alpha of Algorithm 4); after the step, the new pending
    vector is orthogonal to q_0..q_3 (Stephen's trick, eq. 30, for the q_3 component).
    Returns the worst relative deviation."""
    rng = np.random.default_rng(12)
    m = 60
    A = _random_sparse(m, 12)
    Qc, Hc = orc.cgs2_arnoldi(A, rng.standard_normal(m), 4)
    c = rng.standard_normal(3)
    st = cls(A, rng.standard_normal(m), 6)
    st.Q[:, :3] = Qc[:, :3]
    st.H[:3, :2] = Hc[:3, :2]
    st.K[:3, 2] = Hc[:3, 2] - c
    st.k = 3
    st.w = Hc[3, 2] * Qc[:, 3] + Qc[:, :3] @ c
    st.step()
    # the first projection of v = A w (with Stephen's trick) leaves w orthogonal to Q_4
    proj = np.abs(st.Q[:, :4].T @ st.w).max() / np.linalg.norm(st.w)
    st.finish()
    scale = np.abs(Hc).max()
    errs = [proj, abs(st.alphas[-1] - Hc[3, 2]) / Hc[3, 2],
            np.abs(st.Q[:, 3] - Qc[:, 3]).max(),
            np.abs(st.H[:4, 2] - Hc[:4, 2]).max() / scale,
            np.abs(st.H[:5, 3] - Hc[:5, 3]).max() / scale,
            np.abs(st.Q[:, 4] - Qc[:, 4]).max()]
    return max(errs)


def test_crafted_state_exercises_pythagoras_and_stephens_trick():
    assert _crafted_step_errors(orc.DCGS2Arnoldi) < 1e-13


def test_planted_mistakes_are_caught():
    """A wrong sign in Stephen's trick or a dropped representation correction H C / alpha
    only shows at rounding level on well-conditioned runs (both multiply the O(eps)
    coefficient C), so the crafted state with O(1) C is what catches them."""

    class WrongSign(orc.DCGS2Arnoldi):
        def step(self):
            k = self.k
            Qk = self.Q[:, :k]
            w = self.w
            v = self.A @ w
            C = Qk.T @ w
            S = Qk.T @ v
            alpha = np.sqrt(w @ w - C @ C)
            if k >= 1:
                self.H[:k, k - 1] = self.K[:k, k - 1] + C
                self.H[k, k - 1] = alpha
            T = np.empty(k + 1)
            T[:k] = S / alpha
            T[k] = (w @ v + C @ S) / alpha ** 2          # planted: + instead of -
            q = (w - Qk @ C) / alpha
            self.Q[:, k] = q
            self.w = v / alpha - Qk @ T[:k] - q * T[k]
            self.K[:k + 1, k] = T - (self.H[:k + 1, :k] @ C) / alpha
            self.alphas.append(alpha)
            self.k = k + 1
            return alpha

    class NoCorrection(orc.DCGS2Arnoldi):
        def step(self):
            k = self.k
            Qk = self.Q[:, :k]
            w = self.w
            v = self.A @ w
            C = Qk.T @ w
            S = Qk.T @ v
            alpha = np.sqrt(w @ w - C @ C)
            if k >= 1:
                self.H[:k, k - 1] = self.K[:k, k - 1] + C
                self.H[k, k - 1] = alpha
            T = np.empty(k + 1)
            T[:k] = S / alpha
            T[k] = (w @ v - C @ S) / alpha ** 2
            q = (w - Qk @ C) / alpha
            self.Q[:, k] = q
            self.w = v / alpha - Qk @ T[:k] - q * T[k]
            self.K[:k + 1, k] = T                        # planted: correction dropped
            self.alphas.append(alpha)
            self.k = k + 1
            return alpha

    assert _crafted_step_errors(WrongSign) > 1e-3
    assert _crafted_step_errors(NoCorrection) > 1e-3
