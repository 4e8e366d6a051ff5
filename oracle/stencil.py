"""The matrix-free 7-point stencil operator in plain FP64 numpy/scipy (test infrastructure
only: the library never imports it).

The operator is the basis generator of the Arnoldi expansion (Section 4: v = A w on the
unnormalised pending vector) in the form that needs no stored matrix: on an nx x ny x nz
grid (x fastest, row i = ix + nx (iy + ny iz)) with zero values outside it,

    (A x)_i = c0 x_i + c1 x_{i-1} + c2 x_{i+1} + c3 x_{i-nx} + c4 x_{i+nx}
            + c5 x_{i-nx ny} + c6 x_{i+nx ny},

a neighbour term present only when that neighbour lies in the grid.  Two statements of the
same definition, built independently so that one checks the other:

  stencil7_matvec   pads x with one layer of zeros and adds the seven shifted copies
  stencil7_matrix   assembles A as c0 I + sum of Kronecker products of one-dimensional
                    shift matrices (the explicit sparse matrix the Arnoldi oracles take)

Pins (tests/test_oracle_stencil.py): the two statements agree; a loop over every row of a
tiny grid (the definition read literally) agrees with both; the stencil generators in
``synth`` reproduce ``synth.convdiff_csr`` and ``synth.manteuffel_csr`` entry for entry;
the Manteuffel stencil has the closed-form spectrum of Section 6.1.
"""
from __future__ import annotations

import numpy as np


def stencil7_matvec(grid, c, x):
    """y = A x by zero padding and shifted copies."""
    nx, ny, nz = grid
    X = np.asarray(x, dtype=np.float64).reshape(nz, ny, nx)
    P = np.zeros((nz + 2, ny + 2, nx + 2))
    P[1:-1, 1:-1, 1:-1] = X
    core = (slice(1, -1), slice(1, -1), slice(1, -1))
    y = c[0] * P[core]
    y = y + c[1] * P[1:-1, 1:-1, :-2] + c[2] * P[1:-1, 1:-1, 2:]
    y = y + c[3] * P[1:-1, :-2, 1:-1] + c[4] * P[1:-1, 2:, 1:-1]
    y = y + c[5] * P[:-2, 1:-1, 1:-1] + c[6] * P[2:, 1:-1, 1:-1]
    return y.reshape(-1)


def stencil7_matrix(grid, c):
    """A as a scipy CSR matrix: c0 I + c1 (I_z x I_y x L_x) + c2 (I_z x I_y x U_x) + ...,
    where L_n (ones at (i, i-1)) picks the lower neighbour and U_n = L_n^T the upper one."""
    import scipy.sparse as sp
    nx, ny, nz = grid

    def lower(n):
        return sp.eye(n, k=-1, format="csr")

    Ix, Iy, Iz = sp.eye(nx), sp.eye(ny), sp.eye(nz)
    terms = [
        (c[0], sp.kron(Iz, sp.kron(Iy, Ix))),
        (c[1], sp.kron(Iz, sp.kron(Iy, lower(nx)))),
        (c[2], sp.kron(Iz, sp.kron(Iy, lower(nx).T))),
        (c[3], sp.kron(Iz, sp.kron(lower(ny), Ix))),
        (c[4], sp.kron(Iz, sp.kron(lower(ny).T, Ix))),
        (c[5], sp.kron(lower(nz), sp.kron(Iy, Ix))),
        (c[6], sp.kron(lower(nz).T, sp.kron(Iy, Ix))),
    ]
    A = sum(coef * T for coef, T in terms)
    A = sp.csr_matrix(A)
    A.sort_indices()
    return A
