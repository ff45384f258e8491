"""Gradients of L = ||x - x_t||^2 through A(theta) x = b, in plain FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring): the reference for the
differentiable solve of the library.

The adjoint method, written out.  With g = dL/dx = 2 (x - x_t) and lambda
the solution of the transposed system A^T lambda = g:
    dL/db      = lambda,
    dL/dA_ij   = -lambda_i x_j          for every stored entry (i, j),
    dL/dtheta  = sum over stored entries of dL/dA_ij * dA_ij/dtheta.
A(theta) is the 5-point operator of ``workloads.make_vcdiff``:
-div(kappa grad u) + c.grad u on the unit square, kappa = exp(theta) per
cell, an interior face taking the mean of its two cells and a boundary face
its one cell.  Only the diffusion part depends on theta.  A face f with
diffusivity kappa_f contributes kappa_f G_f / h^2 with
G_f = (e_p - e_q)(e_p - e_q)^T for an interior face between cells p and q and
G_f = e_p e_p^T for a boundary face of cell p, so
    lambda^T (dA/dkappa_f) x = (lambda_p - lambda_q)(x_p - x_q) / h^2  (interior)
                             = lambda_p x_p / h^2                      (boundary)
and dkappa_f/dtheta_p = kappa_p / 2 (interior) or kappa_p (boundary).
Dense solves (numpy.linalg.solve) limit it to small grids.
"""
import numpy as np

from workloads.stencils import csr_to_dense, make_vcdiff


def solve_dense(n, theta, b, conv=(10.0, 10.0)):
    """x = A(theta)^{-1} b by dense LU; also returns A (CSR) and its dense copy."""
    A = make_vcdiff(n, theta, conv)
    D = csr_to_dense(A)
    return np.linalg.solve(D, b), A, D


def loss(n, theta, b, x_t, conv=(10.0, 10.0)):
    x, _, _ = solve_dense(n, theta, b, conv)
    return float(np.sum((x - x_t) ** 2))


def gradients(n, theta, b, x_t, conv=(10.0, 10.0)):
    """(L, x, lambda, dL/dvals, dL/dtheta) by the adjoint method."""
    x, A, D = solve_dense(n, theta, b, conv)
    r = x - x_t
    L = float(r @ r)
    lam = np.linalg.solve(D.T, 2.0 * r)
    rows = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.rowptr.astype(np.int64)))
    dvals = -lam[rows] * x[A.col.astype(np.int64)]
    h = 1.0 / (n + 1)
    k = np.exp(theta.reshape(n, n))  # [iy, ix]
    X = x.reshape(n, n)
    Lm = lam.reshape(n, n)
    dth = np.zeros((n, n))
    # x-faces between (iy, i-1) and (iy, i), i = 1 .. n-1
    q = -(Lm[:, 1:] - Lm[:, :-1]) * (X[:, 1:] - X[:, :-1]) / h**2
    dth[:, :-1] += 0.5 * k[:, :-1] * q
    dth[:, 1:] += 0.5 * k[:, 1:] * q
    # y-faces between (iy-1, ix) and (iy, ix)
    q = -(Lm[1:, :] - Lm[:-1, :]) * (X[1:, :] - X[:-1, :]) / h**2
    dth[:-1, :] += 0.5 * k[:-1, :] * q
    dth[1:, :] += 0.5 * k[1:, :] * q
    # boundary faces: left and right columns, bottom and top rows
    bnd = -Lm * X / h**2
    dth[:, 0] += k[:, 0] * bnd[:, 0]
    dth[:, n - 1] += k[:, n - 1] * bnd[:, n - 1]
    dth[0, :] += k[0, :] * bnd[0, :]
    dth[n - 1, :] += k[n - 1, :] * bnd[n - 1, :]
    return L, x, lam, dvals, dth.ravel()
