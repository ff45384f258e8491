"""Differentiable GMRES-SDR solve (the adjoint form): a torch.autograd.Function
whose backward pass solves the transposed system with its own recycle space.

Forward: x = A^{-1} b by GMRES-SDR on the handle ``pair.fwd``.  Backward, given
dL/dx: A^T lambda = dL/dx by GMRES-SDR on ``pair.adj`` (the transposed pattern
is built once per sparsity pattern by sdr_csr_transpose, the values of A^T are
gathered by sdr_gather_values), then dL/db = lambda and dL/dA_ij =
-lambda_i x_j on the stored entries (sdr_value_gradient).  Each handle keeps
its recycle space from one call to the next; when the matrix changes (a new
theta) its SAU is recomputed for the new matrix (exact variant, Section 3.6).
Everything runs in the library's kernels on torch's current stream.
"""
import ctypes

import torch

from .sdr import CSRDevice, Solver, _check, _device_array, _ptr, _stream, load_library, sdr_csr, sdr_solve


class AdjointPair:
    """Forward and transposed GMRES-SDR handles for one sparsity pattern."""

    def __init__(self, n, rowptr: torch.Tensor, col: torch.Tensor, m, k, t, s, zeta=8, seed=231114206,
                 rel_tol=1e-8, max_cycles=200):
        self.n, self.nnz = int(n), int(col.numel())
        self.rowptr = _device_array(rowptr.contiguous(), self.n + 1, "rowptr", torch.int32)
        dev = rowptr.device
        self.col = _device_array(col.contiguous(), self.nnz, "col", torch.int32, dev)
        self.rowptrT = torch.empty(self.n + 1, dtype=torch.int32, device=dev)
        self.colT = torch.empty(self.nnz, dtype=torch.int32, device=dev)
        self.perm = torch.empty(self.nnz, dtype=torch.int32, device=dev)
        work = torch.empty(2 * self.n, dtype=torch.int32, device=dev)
        pat = sdr_csr(self.n, self.nnz, self.rowptr.data_ptr(), self.col.data_ptr(), 0, 0)
        _check(load_library().sdr_csr_transpose(ctypes.byref(pat), _ptr(self.rowptrT), _ptr(self.colT),
                                                _ptr(self.perm), _ptr(work), _stream()), "sdr_csr_transpose")
        torch.cuda.current_stream().synchronize()
        self.fwd = Solver(self.n, m, k, t, s, zeta, seed, rel_tol, max_cycles=max_cycles)
        self.adj = Solver(self.n, m, k, t, s, zeta, seed, rel_tol, max_cycles=max_cycles)
        self._fwd_used = self._adj_used = False
        self.last_stats = {}

    def matrix(self, vals):
        return CSRDevice(self.n, self.rowptr, self.col, vals.contiguous())

    def solve(self, vals: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
        A = self.matrix(vals)
        if self._fwd_used:
            self.fwd.recycle(A, 0)
        x = torch.zeros_like(b, memory_format=torch.contiguous_format)
        _, self.last_stats["forward"] = sdr_solve(self.fwd.h, A, b.contiguous(), x)
        self._fwd_used = True
        return x

    def solve_adjoint(self, vals: torch.Tensor, g: torch.Tensor) -> torch.Tensor:
        vals = _device_array(vals.contiguous(), self.nnz, "vals", device=self.perm.device)
        valsT = torch.empty_like(vals)
        _check(load_library().sdr_gather_values(_ptr(vals), _ptr(self.perm), self.nnz, _ptr(valsT),
                                                _stream()), "sdr_gather_values")
        AT = CSRDevice(self.n, self.rowptrT, self.colT, valsT)
        if self._adj_used:
            self.adj.recycle(AT, 0)
        lam = torch.zeros_like(g, memory_format=torch.contiguous_format)
        _, self.last_stats["adjoint"] = sdr_solve(self.adj.h, AT, g.contiguous(), lam)
        self._adj_used = True
        return lam

    def value_gradient(self, vals, lam, x):
        A = self.matrix(vals).c_struct()
        lam = _device_array(lam.contiguous(), self.n, "lambda", device=self.perm.device)
        x = _device_array(x.contiguous(), self.n, "x", device=self.perm.device)
        grad = torch.empty_like(vals, memory_format=torch.contiguous_format)  # nnz entries: c_struct checked
        _check(load_library().sdr_value_gradient(ctypes.byref(A), _ptr(lam), _ptr(x), _ptr(grad), _stream()),
               "sdr_value_gradient")
        return grad

    def close(self):
        self.fwd.close()
        self.adj.close()


class SDRSolve(torch.autograd.Function):
    """x = A^{-1} b, differentiable in the stored values of A and in b."""

    @staticmethod
    def forward(ctx, vals, b, pair):
        x = pair.solve(vals.detach(), b.detach())
        ctx.pair = pair
        ctx.save_for_backward(vals.detach(), x)
        return x

    @staticmethod
    def backward(ctx, gx):
        vals, x = ctx.saved_tensors
        lam = ctx.pair.solve_adjoint(vals, gx.contiguous())
        gvals = ctx.pair.value_gradient(vals, lam, x) if ctx.needs_input_grad[0] else None
        gb = lam if ctx.needs_input_grad[1] else None
        return gvals, gb, None


def solve(vals: torch.Tensor, b: torch.Tensor, pair: AdjointPair) -> torch.Tensor:
    return SDRSolve.apply(vals, b, pair)
