"""Synthetic sparse operators in CSR form (int32 indices, float64 values).

The paper's own Krylov experiments use the Manteuffel "central differences" matrix
(Section 6.1, its eigenvalue formula) and SuiteSparse / 3D Laplace problems that are not
available here.  The throughput workloads are therefore convection-diffusion operators

    -div(kappa grad u) + b . grad u      on (0,1)^d, homogeneous Dirichlet boundary,

discretised on N interior points per direction (h = 1/(N+1), lexicographic order with x
fastest), with

  * diffusion: the 5-point (2D) / 7-point (3D) stencil, face coefficient = harmonic mean of
    the two nodal kappas (a boundary face uses the interior node's kappa);
  * convection: first-order upwind in every direction (gives an M-matrix);
  * every row scaled by h^2.

Within a row the column indices are strictly increasing.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """Host CSR matrix: row_ptr int32[m+1], col_idx int32[nnz], val float64[nnz]."""
    m: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.m, self.m))


def _assemble(m: int, offsets, values, masks) -> CSR:
    """Stack per-stencil-point value/mask arrays (already in increasing column order)."""
    vals = np.stack(values, axis=1)            # (m, p)
    mask = np.stack(masks, axis=1)             # (m, p)
    counts = mask.sum(axis=1, dtype=np.int64)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 indices")
    rows = np.arange(m, dtype=np.int64)
    cols = rows[:, None] + np.asarray(offsets, dtype=np.int64)[None, :]
    col_idx = cols[mask].astype(np.int32)
    val = vals[mask].astype(np.float64)
    return CSR(m, row_ptr.astype(np.int32), col_idx, val)


def convdiff_csr(N: int, dim: int, wind, kappa=None) -> CSR:
    """Upwind convection-diffusion on an N^dim grid (rows scaled by h^2).

    wind:  a constant vector of length ``dim`` or a nodal field of shape (dim, N, ..., N)
           with axis order (z, y, x) for the spatial part (x fastest in memory).
    kappa: None (kappa = 1) or a nodal field of shape (N,)*dim, positive.
    """
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    h = 1.0 / (N + 1)
    shape = (N,) * dim
    m = N ** dim
    if kappa is None:
        kap = np.ones(shape)
    else:
        kap = np.asarray(kappa, dtype=np.float64).reshape(shape)
    wind = np.asarray(wind, dtype=np.float64)
    if wind.ndim == 1:
        bfield = [np.full(shape, wind[a]) for a in range(dim)]   # a = 0 -> x, 1 -> y, 2 -> z
    else:
        bfield = [wind[a].reshape(shape) for a in range(dim)]
    diag = np.zeros(shape)
    lower = {}   # axis -> coefficient of the (i-1) neighbour
    upper = {}
    for a in range(dim):              # a = 0 is x (last numpy axis), 1 is y, 2 is z
        ax = dim - 1 - a
        # face coefficients towards the lower / upper neighbour along this axis
        kl = kap.copy()
        ku = kap.copy()
        sl_hi = [slice(None)] * dim
        sl_lo = [slice(None)] * dim
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(None, -1)
        harm = 2.0 * kap[tuple(sl_hi)] * kap[tuple(sl_lo)] / (kap[tuple(sl_hi)] + kap[tuple(sl_lo)])
        kl[tuple(sl_hi)] = harm
        ku[tuple(sl_lo)] = harm
        b = bfield[a]
        bpos = np.maximum(b, 0.0) * h
        bneg = np.maximum(-b, 0.0) * h
        diag += kl + ku + bpos + bneg
        lo = -(kl + bpos)
        up = -(ku + bneg)
        # neighbours outside the grid are Dirichlet boundary nodes: drop them
        idx_first = [slice(None)] * dim
        idx_first[ax] = 0
        idx_last = [slice(None)] * dim
        idx_last[ax] = N - 1
        mlo = np.ones(shape, dtype=bool)
        mup = np.ones(shape, dtype=bool)
        mlo[tuple(idx_first)] = False
        mup[tuple(idx_last)] = False
        lower[a] = (lo, mlo)
        upper[a] = (up, mup)
    stride = [1, N, N * N]
    offsets, values, masks = [], [], []
    for a in reversed(range(dim)):        # z-, y-, x- neighbours (increasing column)
        offsets.append(-stride[a])
        values.append(lower[a][0].reshape(m))
        masks.append(lower[a][1].reshape(m))
    offsets.append(0)
    values.append(diag.reshape(m))
    masks.append(np.ones(m, dtype=bool))
    for a in range(dim):                  # x+, y+, z+ neighbours
        offsets.append(stride[a])
        values.append(upper[a][0].reshape(m))
        masks.append(upper[a][1].reshape(m))
    return _assemble(m, offsets, values, masks)


def manteuffel_csr(k: int, beta: float = 0.5) -> CSR:
    """Manteuffel's central-difference matrix on a k x k grid with h = 1 (Section 6.1).

    A = I (x) T + T (x) I with T = tridiag(-1 - beta/2, 2, -1 + beta/2): the 5-point
    Laplacian M plus (beta/2) times the skew-symmetric centred first difference N.  Its
    eigenvalues are 2[2 - sqrt(1-(beta/2)^2)(cos(l pi/(k+1)) + cos(j pi/(k+1)))].
    """
    m = k * k
    lo = -1.0 - beta / 2.0
    up = -1.0 + beta / 2.0
    shape = (k, k)
    offsets, values, masks = [], [], []
    ones = np.ones(m)
    grid_y, grid_x = np.meshgrid(np.arange(k), np.arange(k), indexing="ij")
    gx = grid_x.reshape(m)
    gy = grid_y.reshape(m)
    for off, v, msk in ((-k, lo, gy > 0), (-1, lo, gx > 0), (0, 4.0, np.ones(m, bool)),
                        (1, up, gx < k - 1), (k, up, gy < k - 1)):
        offsets.append(off)
        values.append(v * ones)
        masks.append(msk)
    del shape
    return _assemble(m, offsets, values, masks)


@dataclass
class Stencil7:
    """Constant-coefficient 7-point stencil on an nx x ny x nz grid (x fastest), zero outside.

    c = (centre, x-1, x+1, y-1, y+1, z-1, z+1): row i = ix + nx (iy + ny iz) has c[0] on the
    diagonal and each neighbour coefficient where that neighbour lies in the grid."""
    grid: tuple
    c: tuple

    @property
    def m(self) -> int:
        nx, ny, nz = self.grid
        return nx * ny * nz

    @property
    def nnz(self) -> int:
        """Number of stored entries of the equivalent CSR matrix (zero coefficients count)."""
        nx, ny, nz = self.grid
        m = self.m
        return m + 2 * (m - ny * nz) + 2 * (m - nx * nz) + 2 * (m - nx * ny)


def convdiff_stencil7(N: int, dim: int, wind) -> Stencil7:
    """The operator of ``convdiff_csr(N, dim, wind)`` with kappa = 1 and a constant wind, as a
    stencil.  Every row of that matrix carries the same coefficients (the harmonic mean of
    two unit kappas is 1, and a boundary face uses the interior kappa 1), so the stencil
    with zero values outside the grid is the same matrix; the coefficients are formed by the
    same floating-point expressions, so they equal the CSR values bit for bit."""
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    h = 1.0 / (N + 1)
    wind = np.asarray(wind, dtype=np.float64)
    diag = 0.0
    lo = [0.0, 0.0, 0.0]
    up = [0.0, 0.0, 0.0]
    for a in range(dim):
        kl = ku = 1.0
        bpos = max(float(wind[a]), 0.0) * h
        bneg = max(-float(wind[a]), 0.0) * h
        diag += kl + ku + bpos + bneg
        lo[a] = -(kl + bpos)
        up[a] = -(ku + bneg)
    grid = (N, N, N) if dim == 3 else (N, N, 1)
    return Stencil7(grid, (diag, lo[0], up[0], lo[1], up[1], lo[2], up[2]))


def manteuffel_stencil7(k: int, beta: float = 0.5) -> Stencil7:
    """``manteuffel_csr(k, beta)`` as a 5-point stencil on a k x k grid (nz = 1)."""
    lo = -1.0 - beta / 2.0
    up = -1.0 + beta / 2.0
    return Stencil7((k, k, 1), (4.0, lo, up, lo, up, 0.0, 0.0))


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def config1_operator() -> CSR:
    """2D, N = 100, constant wind along (1,1), Peclet 10 (|b| = 10), kappa = 1."""
    return convdiff_csr(100, 2, 10.0 * _unit([1.0, 1.0]))


def config2_operator(N: int = 252) -> CSR:
    """3D, N = 252 (m = 16,003,008), constant wind along (1, 0.5, 0.25), Peclet 50."""
    return convdiff_csr(N, 3, 50.0 * _unit([1.0, 0.5, 0.25]))


def config1_stencil() -> Stencil7:
    """``config1_operator()`` in matrix-free form."""
    return convdiff_stencil7(100, 2, 10.0 * _unit([1.0, 1.0]))


def config2_stencil(N: int = 252) -> Stencil7:
    """``config2_operator(N)`` in matrix-free form."""
    return convdiff_stencil7(N, 3, 50.0 * _unit([1.0, 0.5, 0.25]))


def config3_operator(N: int = 1000, seed: int = 1003) -> CSR:
    """2D, kappa i.i.d. log-uniform on [0.1, 10] (seeded), wind along (1,1), Peclet 100."""
    rng = np.random.default_rng(seed)
    kappa = 10.0 ** rng.uniform(-1.0, 1.0, size=(N, N))
    return convdiff_csr(N, 2, 100.0 * _unit([1.0, 1.0]), kappa=kappa)


def varcoef_fields_2d(N: int, seed: int, corr_len: float = 0.05, pe: float = 100.0,
                      n_modes: int = 8):
    """Log-normal kappa (sigma = 1) and a divergence-free smooth wind, both seeded.

    kappa = exp(g): g is white noise smoothed by a Gaussian of correlation length
    ``corr_len`` (periodic FFT convolution), renormalised to zero mean and unit variance.
    wind = curl of a stream function made of ``n_modes`` random sine modes, scaled so that
    max |b| = pe.  Returns (kappa (N,N), wind (2,N,N)) with wind[0] = b_x, wind[1] = b_y.
    """
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((N, N))
    f = np.fft.fftfreq(N, d=1.0 / (N + 1))
    fy, fx = np.meshgrid(f, f, indexing="ij")
    kern = np.exp(-2.0 * (np.pi * corr_len) ** 2 * (fx ** 2 + fy ** 2))
    g = np.real(np.fft.ifft2(np.fft.fft2(noise) * kern))
    g = (g - g.mean()) / g.std()
    kappa = np.exp(g)
    h = 1.0 / (N + 1)
    xs = h * np.arange(1, N + 1)
    Y, X = np.meshgrid(xs, xs, indexing="ij")
    bx = np.zeros((N, N))
    by = np.zeros((N, N))
    for _ in range(n_modes):
        kx, ky = rng.integers(1, 5, size=2)
        amp = rng.standard_normal()
        ph = rng.uniform(0, 2 * np.pi, size=2)
        sx = np.sin(np.pi * kx * X + ph[0])
        cx = np.cos(np.pi * kx * X + ph[0])
        sy = np.sin(np.pi * ky * Y + ph[1])
        cy = np.cos(np.pi * ky * Y + ph[1])
        # psi = amp sx sy ; b = (d psi/dy, -d psi/dx)
        bx += amp * sx * (np.pi * ky) * cy
        by += -amp * (np.pi * kx) * cx * sy
    scale = pe / np.sqrt(bx ** 2 + by ** 2).max()
    return kappa, np.stack([bx * scale, by * scale])


def config5_operator(N: int = 1024, seed: int = 64) -> CSR:
    """2D variable-coefficient operator of the learned-preconditioner family."""
    kappa, wind = varcoef_fields_2d(N, seed)
    return convdiff_csr(N, 2, wind, kappa=kappa)
