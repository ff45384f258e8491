"""The refined form (float32 inner GMRES-SDR inside float64 iterative
refinement) against the FP64 oracle.

The inner solver keeps V, U, the SpMV, the window dots and the Arnoldi update
in float32 with float32 accumulation; the sketched QR, the harmonic-Ritz
eigenproblem and the outer residual r = b - A x stay float64.  Bars: the true
residual, recomputed on the host in FP64 with the oracle's SpMV, is below the
requested 1e-10 ||b||, and the solution lies within 1e-8 relative of the
oracle's FP64 GMRES-SDR solution at rel_tol 1e-12.
"""
import numpy as np
import pytest

import workloads as W
from oracle import sdr as osdr
from oracle.sketch import SparseSign

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 231114206


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2311_14206_gb300 as P
    return P


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def test_refined_sequence_matches_fp64_oracle(P):
    A0 = W.make_cd3d(20, (20.0, 10.0, 5.0))
    dvec = W.diag_perturbation(A0.n)
    As = list(W.sequence_matrices(A0, 3, 1e-3, dvec))
    bs = [W.rhs(A0.n, i) for i in range(3)]
    m, k, t, s, zeta = 40, 10, 2, 120, 8
    solver = P.Solver(A0.n, m, k, t, s, zeta, SEED, 1e-10, max_cycles=8, precision=P.SDR_PREC_F32_REFINED,
                      inner_rel_tol=1e-4)
    S = SparseSign(SEED, A0.n, s, zeta)
    for i, (A, b) in enumerate(zip(As, bs)):
        Ad = P.CSRDevice.from_numpy(A, with_f32=True)
        if i > 0:
            solver.recycle(Ad, 0)
        x, st, stats = solver.solve(Ad, dev(b))
        xh = x.cpu().numpy()
        bn = np.linalg.norm(b)
        relres = np.linalg.norm(b - osdr.csr_matvec(A, xh)) / bn
        ref = osdr.solve(A, b, S, m=m, k=k, t=t, rel_tol=1e-12)
        err = np.linalg.norm(xh - ref.x) / np.linalg.norm(ref.x)
        print(f"system {i}: refinements {stats['refinements']} inner cycles {stats['cycles']} "
              f"rel res {relres:.2e} error vs oracle {err:.2e}")
        assert st == 0 and stats["converged"] == 1
        assert stats["refinements"] >= 1
        assert relres <= 1e-10
        assert err <= 1e-8
    solver.close()


def test_refined_needs_float32_values(P):
    A = W.make_cd2d(16)
    solver = P.Solver(A.n, 20, 4, 2, 40, 8, SEED, 1e-10, precision=P.SDR_PREC_F32_REFINED)
    with pytest.raises(P.SdrError):
        solver.solve(P.CSRDevice.from_numpy(A), dev(W.rhs(A.n)))
    solver.close()


def test_refined_already_converged(P):
    A = W.make_cd2d(16)
    b = W.rhs(A.n)
    xs = np.linalg.solve(W.csr_to_dense(A), b)
    solver = P.Solver(A.n, 20, 4, 2, 40, 8, SEED, 1e-10, precision=P.SDR_PREC_F32_REFINED)
    xd = dev(xs)
    st, stats = P.sdr_solve(solver.h, P.CSRDevice.from_numpy(A, with_f32=True), dev(b), xd)
    assert st == 0 and stats["refinements"] == 0 and stats["cycles"] == 0
    solver.close()
