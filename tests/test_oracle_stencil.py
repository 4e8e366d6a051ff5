"""Pins of the stencil oracle (CPU): the two statements of the definition against each
other and against a literal loop, the generators in synth against the CSR generators, and
the Manteuffel stencil against its closed-form spectrum (Section 6.1)."""
import numpy as np
import pytest

import synth
from oracle.stencil import stencil7_matrix, stencil7_matvec


def literal_matvec(grid, c, x):
    """The definition read literally: one row at a time, each neighbour if it exists."""
    nx, ny, nz = grid
    y = np.zeros(nx * ny * nz)
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                i = ix + nx * (iy + ny * iz)
                acc = c[0] * x[i]
                if ix > 0:
                    acc += c[1] * x[i - 1]
                if ix < nx - 1:
                    acc += c[2] * x[i + 1]
                if iy > 0:
                    acc += c[3] * x[i - nx]
                if iy < ny - 1:
                    acc += c[4] * x[i + nx]
                if iz > 0:
                    acc += c[5] * x[i - nx * ny]
                if iz < nz - 1:
                    acc += c[6] * x[i + nx * ny]
                y[i] = acc
    return y


@pytest.mark.parametrize("grid", [(1, 1, 1), (5, 1, 1), (1, 4, 3), (3, 2, 4), (6, 5, 1),
                                  (4, 4, 4)])
def test_two_statements_and_literal_loop_agree(grid):
    rng = np.random.default_rng(sum(grid))
    c = rng.standard_normal(7)
    x = rng.standard_normal(int(np.prod(grid)))
    ref = literal_matvec(grid, c, x)
    scale = np.abs(c).sum() * np.abs(x).max()
    assert np.abs(stencil7_matvec(grid, c, x) - ref).max() <= 1e-15 * scale
    assert np.abs(stencil7_matrix(grid, c) @ x - ref).max() <= 1e-15 * scale


def test_each_coefficient_hits_one_neighbour():
    # a single nonzero coefficient must move a unit impulse to exactly one place
    grid = (5, 4, 3)
    nx, ny, nz = grid
    centre = 2 + nx * (1 + ny * 1)
    x = np.zeros(nx * ny * nz)
    x[centre] = 1.0
    # row r receives x_{r+d} through coefficient j, so the impulse lands at centre - d
    offsets = [0, -1, 1, -nx, nx, -nx * ny, nx * ny]
    for j, d in enumerate(offsets):
        c = np.zeros(7)
        c[j] = 1.0
        y = stencil7_matvec(grid, c, x)
        assert np.flatnonzero(y).tolist() == [centre - d]


@pytest.mark.parametrize("N,dim", [(7, 3), (9, 2)])
def test_convdiff_stencil_is_the_csr_matrix(N, dim):
    wind = (50.0 * np.array([1.0, 0.5, 0.25]) / np.linalg.norm([1.0, 0.5, 0.25]))[:dim]
    st = synth.convdiff_stencil7(N, dim, wind)
    A = synth.convdiff_csr(N, dim, wind).to_scipy()
    B = stencil7_matrix(st.grid, st.c)
    B.eliminate_zeros()
    assert (A != B).nnz == 0                       # entry for entry, bit for bit
    assert st.nnz == A.nnz


def test_config_stencils_match_config_operators():
    for st, A in ((synth.config1_stencil(), synth.config1_operator()),
                  (synth.config2_stencil(10), synth.config2_operator(10))):
        B = stencil7_matrix(st.grid, st.c)
        B.eliminate_zeros()
        assert (A.to_scipy() != B).nnz == 0


def test_manteuffel_stencil_matrix_and_spectrum():
    k, beta = 6, 0.5
    st = synth.manteuffel_stencil7(k, beta)
    B = stencil7_matrix(st.grid, st.c)
    B.eliminate_zeros()
    assert (synth.manteuffel_csr(k, beta).to_scipy() != B).nnz == 0
    # Section 6.1: 2 [2 - sqrt(1 - (beta/2)^2) (cos(l pi/(k+1)) + cos(j pi/(k+1)))]
    t = np.cos(np.arange(1, k + 1) * np.pi / (k + 1))
    exact = np.sort((2 * (2 - np.sqrt(1 - (beta / 2) ** 2) * (t[:, None] + t[None, :]))).ravel())
    ev = np.linalg.eigvals(B.toarray())
    assert np.abs(ev.imag).max() < 1e-10
    assert np.allclose(np.sort(ev.real), exact, atol=1e-10)
