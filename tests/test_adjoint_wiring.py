"""The autograd wiring of the differentiable solve (SDRSolve) on CPU.

SDRSolve's forward calls pair.solve and its backward pair.solve_adjoint and
pair.value_gradient; on the GPU those are GMRES-SDR solves and library
kernels.  Here a dense stand-in supplies the same three operations (x = A^-1 b,
lambda = A^-T g, -lambda_i x_j on the stored entries), so torch's gradcheck
checks what SDRSolve itself does: which tensors it saves, which inputs get a
gradient and the order of the returned gradients."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W  # noqa: E402
from paper_2311_14206_gb300.adjoint import SDRSolve  # noqa: E402


class DensePair:
    def __init__(self, A):
        self.n = A.n
        self.rows = torch.as_tensor(np.repeat(np.arange(A.n), np.diff(A.rowptr.astype(np.int64))))
        self.col = torch.as_tensor(A.col.astype(np.int64))

    def dense(self, vals):
        M = torch.zeros(self.n, self.n, dtype=vals.dtype)
        M[self.rows, self.col] = vals
        return M

    def solve(self, vals, b):
        return torch.linalg.solve(self.dense(vals), b)

    def solve_adjoint(self, vals, g):
        return torch.linalg.solve(self.dense(vals).T, g)

    def value_gradient(self, vals, lam, x):
        return -lam[self.rows] * x[self.col]


def test_sdrsolve_gradients_match_finite_differences():
    A = W.make_cd2d(5, (3.0, -2.0))
    pair = DensePair(A)
    vals = torch.tensor(A.val, dtype=torch.float64, requires_grad=True)
    b = torch.tensor(W.rhs(A.n, 3), dtype=torch.float64, requires_grad=True)
    # scale the values so that finite differences of the solution are well conditioned
    f = lambda v, bb: SDRSolve.apply(v * 1e-2, bb, pair)  # noqa: E731
    assert torch.autograd.gradcheck(f, (vals, b), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_sdrsolve_gradient_only_where_asked():
    A = W.make_cd2d(4)
    pair = DensePair(A)
    vals = torch.tensor(A.val, dtype=torch.float64, requires_grad=True)
    b = torch.tensor(W.rhs(A.n, 1), dtype=torch.float64)  # no gradient wanted for b
    x = SDRSolve.apply(vals, b, pair)
    (x * x).sum().backward()
    assert vals.grad is not None and b.grad is None
    # dL/dA_ij = -lambda_i x_j with A^T lambda = dL/dx = 2x
    xd = x.detach()
    lam = torch.linalg.solve(pair.dense(vals.detach()).T, 2 * xd)
    assert torch.allclose(vals.grad, -lam[pair.rows] * xd[pair.col], rtol=1e-12, atol=1e-15)
