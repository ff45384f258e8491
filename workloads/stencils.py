"""Finite-difference convection-diffusion operators in CSR form.

The paper's test family is the convection-diffusion operator of its Section 6.3
(a 2D Kronecker-sum form with central differences).  The synthetic workloads
use the same family with first-order upwind convection on 2D and 3D grids and
a variable-coefficient 2D variant.  Grid points are ordered lexicographically
with x fastest; a row's entries are stored with ascending column index.

Unit square/cube, h = 1/(n+1), homogeneous Dirichlet boundary (neighbours
outside the grid are dropped).
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """Square sparse matrix: int32 row pointers/columns, float64 values."""

    n: int
    rowptr: np.ndarray  # int32 [n+1]
    col: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def copy(self) -> "CSR":
        return CSR(self.n, self.rowptr.copy(), self.col.copy(), self.val.copy())


def _assemble(n_rows: int, offsets, cols, vals, valid) -> CSR:
    """Pack per-offset column/value/validity arrays (shape [n_rows, n_off],
    offsets in ascending column order) into CSR."""
    counts = valid.sum(axis=1)
    rowptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 range")
    col = cols[valid].astype(np.int32)
    val = vals[valid].astype(np.float64)
    return CSR(n_rows, rowptr.astype(np.int32), col, val)


def _upwind_stencil(n: int, dim: int, conv, diff=1.0):
    """Coefficients of -diff*Lap_h u + c.grad_h u with first-order upwind
    convection (backward difference when c_i > 0, forward when c_i < 0)."""
    h = 1.0 / (n + 1)
    diag = 2.0 * dim * diff / h**2 + sum(abs(float(c)) for c in conv) / h
    lower = []  # coefficient of u_{p - e_i}
    upper = []  # coefficient of u_{p + e_i}
    for c in conv:
        c = float(c)
        lower.append(-diff / h**2 - max(c, 0.0) / h)
        upper.append(-diff / h**2 + min(c, 0.0) / h)
    return diag, lower, upper


def make_cd2d(n: int, conv=(10.0, 10.0), diff: float = 1.0) -> CSR:
    """5-point upwind convection-diffusion on an n x n grid (N = n^2)."""
    diag, lo, up = _upwind_stencil(n, 2, conv, diff)
    N = n * n
    p = np.arange(N, dtype=np.int64)
    ix, iy = p % n, p // n
    offs = [-n, -1, 0, 1, n]
    ok = [iy > 0, ix > 0, np.ones(N, bool), ix < n - 1, iy < n - 1]
    coef = [lo[1], lo[0], diag, up[0], up[1]]
    cols = np.stack([p + o for o in offs], axis=1)
    vals = np.broadcast_to(np.array(coef, dtype=np.float64), (N, 5))
    return _assemble(N, offs, cols, vals, np.stack(ok, axis=1))


def make_cd3d(n: int, conv=(20.0, 10.0, 5.0), diff: float = 1.0) -> CSR:
    """7-point upwind convection-diffusion on an n^3 grid (N = n^3).

    Built plane by plane to bound the temporary memory at large n."""
    diag, lo, up = _upwind_stencil(n, 3, conv, diff)
    n2 = n * n
    N = n2 * n
    coef = np.array([lo[2], lo[1], lo[0], diag, up[0], up[1], up[2]], dtype=np.float64)
    offs = np.array([-n2, -n, -1, 0, 1, n, n2], dtype=np.int64)
    # counts per row, then fill plane by plane
    q = np.arange(n2, dtype=np.int64)
    ix, iy = q % n, q // n
    inplane = np.stack([np.ones(n2, bool), iy > 0, ix > 0, np.ones(n2, bool),
                        ix < n - 1, iy < n - 1, np.ones(n2, bool)], axis=1)
    rowptr = np.zeros(N + 1, dtype=np.int64)
    counts_plane = []
    for iz in range(n):
        v = inplane.copy()
        v[:, 0] &= iz > 0
        v[:, 6] &= iz < n - 1
        counts_plane.append(v)
    nnz = 0
    cnt = np.empty(N, dtype=np.int64)
    for iz in range(n):
        cnt[iz * n2:(iz + 1) * n2] = counts_plane[iz].sum(axis=1)
    np.cumsum(cnt, out=rowptr[1:])
    nnz = int(rowptr[-1])
    if nnz >= 2**31:
        raise ValueError("nnz exceeds int32 range")
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    for iz in range(n):
        v = counts_plane[iz]
        p = iz * n2 + q
        cols = p[:, None] + offs[None, :]
        a, b = rowptr[iz * n2], rowptr[(iz + 1) * n2]
        col[a:b] = cols[v].astype(np.int32)
        val[a:b] = np.broadcast_to(coef, (n2, 7))[v]
    return CSR(N, rowptr.astype(np.int32), col, val)


def make_cd_paper(n: int, alpha: float) -> CSR:
    """The paper's Section 6.3 operator (L (x) I + I (x) L) + alpha (D (x) I + I (x) D)
    with L = (n+1)^2 tridiag(1, -2, 1) and D = (n+1)/2 tridiag(-1, 0, 1)."""
    N = n * n
    l_off, l_diag = (n + 1) ** 2, -2.0 * (n + 1) ** 2
    d_sub, d_sup = -(n + 1) / 2.0, (n + 1) / 2.0
    p = np.arange(N, dtype=np.int64)
    ix, iy = p % n, p // n
    offs = [-n, -1, 0, 1, n]
    ok = [iy > 0, ix > 0, np.ones(N, bool), ix < n - 1, iy < n - 1]
    coef = [l_off + alpha * d_sub, l_off + alpha * d_sub, 2 * l_diag,
            l_off + alpha * d_sup, l_off + alpha * d_sup]
    cols = np.stack([p + o for o in offs], axis=1)
    vals = np.broadcast_to(np.array(coef, dtype=np.float64), (N, 5))
    return _assemble(N, offs, cols, vals, np.stack(ok, axis=1))


def vcdiff_faces(n: int, theta: np.ndarray):
    """Face diffusivities of the variable-coefficient operator.

    kappa = exp(theta) per cell; an interior face takes the arithmetic mean of
    its two cells, a boundary face the value of its one cell.  Returns
    (kx, ky) with kx[iy, i] the face between x-cells i-1 and i (i = 0..n, the
    two ends being boundary faces) and ky[i, ix] likewise in y."""
    k = np.exp(theta.reshape(n, n))  # [iy, ix]
    kx = np.empty((n, n + 1))
    kx[:, 1:n] = 0.5 * (k[:, :-1] + k[:, 1:])
    kx[:, 0] = k[:, 0]
    kx[:, n] = k[:, n - 1]
    ky = np.empty((n + 1, n))
    ky[1:n, :] = 0.5 * (k[:-1, :] + k[1:, :])
    ky[0, :] = k[0, :]
    ky[n, :] = k[n - 1, :]
    return kx, ky


def make_vcdiff(n: int, theta: np.ndarray, conv=(10.0, 10.0)) -> CSR:
    """5-point -div(kappa grad u) + c.grad u with kappa = exp(theta) per cell
    (face values from ``vcdiff_faces``) and upwind convection."""
    h = 1.0 / (n + 1)
    kx, ky = vcdiff_faces(n, theta)
    cx, cy = float(conv[0]), float(conv[1])
    N = n * n
    west = -kx[:, :n] / h**2 - max(cx, 0.0) / h  # coefficient of u_{p-1}
    east = -kx[:, 1:] / h**2 + min(cx, 0.0) / h  # coefficient of u_{p+1}
    south = -ky[:n, :] / h**2 - max(cy, 0.0) / h
    north = -ky[1:, :] / h**2 + min(cy, 0.0) / h
    diag = (kx[:, :n] + kx[:, 1:] + ky[:n, :] + ky[1:, :]) / h**2 + (abs(cx) + abs(cy)) / h
    p = np.arange(N, dtype=np.int64)
    ix, iy = p % n, p // n
    offs = [-n, -1, 0, 1, n]
    ok = [iy > 0, ix > 0, np.ones(N, bool), ix < n - 1, iy < n - 1]
    cols = np.stack([p + o for o in offs], axis=1)
    vals = np.stack([south.ravel(), west.ravel(), diag.ravel(), east.ravel(), north.ravel()], axis=1)
    return _assemble(N, offs, cols, vals, np.stack(ok, axis=1))


def perturb_diag(A: CSR, dvec: np.ndarray, scale: float) -> CSR:
    """A + scale * diag(dvec) (the diagonal entry is present in every row)."""
    B = A.copy()
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.rowptr.astype(np.int64)))
    on_diag = A.col.astype(np.int64) == rows
    if on_diag.sum() != A.n:
        raise ValueError("every row needs a stored diagonal entry")
    B.val[on_diag] += scale * dvec[rows[on_diag]]
    return B


def csr_transpose(A: CSR) -> CSR:
    """Transpose in CSR form (columns ascending within a row)."""
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.rowptr.astype(np.int64)))
    order = np.lexsort((rows, A.col.astype(np.int64)))
    col_t = rows[order].astype(np.int32)
    val_t = A.val[order]
    counts = np.bincount(A.col.astype(np.int64), minlength=A.n)
    rowptr = np.zeros(A.n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(A.n, rowptr.astype(np.int32), col_t, val_t)


def csr_to_dense(A: CSR) -> np.ndarray:
    D = np.zeros((A.n, A.n))
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr.astype(np.int64)))
    np.add.at(D, (rows, A.col.astype(np.int64)), A.val)
    return D
