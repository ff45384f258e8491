"""Parity of the refined form at its own size: the 3D convection-diffusion
sequence on a 256^3 grid (N = 16,777,216, 117 M nonzeros), m = 80, k = 20,
t = 2, s = 400, zeta = 8, float32 inner solves inside float64 iterative
refinement to a true relative residual of 1e-10 (the precision workload).

A whole solve at this size is out of the oracle's reach; checked instead:
  * the first inner solve's first 8 sketched residuals against the oracle's
    first 8 steps of Algorithm 1 on the same right-hand side (b rounded to
    float32, x0 = 0) in float64.  The inner solver stores its basis and runs
    its SpMV in float32, so the bar is the float32 level: 1e-4 relative
    (eight steps of float32 rounding, 2^-24 per operation, amplified by the
    Arnoldi recurrence), against 1e-8 for the float64 path;
  * the true residual ||b - A x|| of every solve, recomputed on the host in
    float64, below 1e-10 ||b|| (up to the rounding of that recomputation);
  * the exact recycle to the next matrix and a second refined solve from it."""
import numpy as np
import pytest

import bench
import workloads as W
from oracle import sdr as osdr
from oracle.sketch import SparseSign

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps
STEPS = 8


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2311_14206_gb300 as P
    return P


def assert_true_residual(A, b, x, tol_rel):
    r = b - osdr.csr_matvec(A, x)
    absA = W.CSR(A.n, A.rowptr, A.col, np.abs(A.val))
    slack = 16 * EPS * np.linalg.norm(osdr.csr_matvec(absA, np.abs(x)))
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert np.linalg.norm(r) <= tol_rel * np.linalg.norm(b) + slack, rel
    return rel


def test_refined_form_full_size(P):
    cfg = bench.F32IR
    A0, dvec, diag_pos = bench.make_inputs(cfg)
    N = A0.n
    assert N == 256 ** 3
    m, k, t, s, zeta, rel_tol = cfg["m"], cfg["k"], cfg["t"], cfg["s"], cfg["zeta"], cfg["rel_tol"]
    As = [W.CSR(N, A0.rowptr, A0.col, bench.system_values(A0, dvec, diag_pos, i, cfg["eps"])) for i in (1, 2)]
    bs = [W.rhs(N, i) for i in (0, 1)]
    solver = P.Solver(N, m, k, t, s, zeta, cfg["seed"], rel_tol, precision=P.SDR_PREC_F32_REFINED,
                      inner_rel_tol=cfg["inner_rel_tol"])
    try:
        mats = []
        for A in As:
            val = torch.as_tensor(A.val, device="cuda")
            mats.append(P.CSRDevice(N, torch.as_tensor(A.rowptr, device="cuda"), torch.as_tensor(A.col, device="cuda"),
                                    val, val.to(torch.float32)))
        x1, st, stats = solver.solve(mats[0], torch.as_tensor(bs[0], device="cuda"))
        assert st == 0 and stats["converged"] == 1 and stats["refinements"] >= 1, stats
        sres, _ = solver.history()
        assert_true_residual(As[0], bs[0], x1.cpu().numpy(), rel_tol)
        # the first inner solve: A d = float32(b), d0 = 0, against the float64 oracle
        b32 = bs[0].astype(np.float32).astype(np.float64)
        S = SparseSign(cfg["seed"], N, s, zeta)
        ref = osdr.cycle(As[0], b32, None, None, None, S, 0.0, STEPS, t, k)
        g = np.asarray(sres[:STEPS])
        r = np.asarray(ref.sres[:STEPS])
        bn = np.linalg.norm(b32)
        assert np.all(np.abs(g - r) <= 1e-4 * r + 1e-7 * bn), (g, r)
        del S
        # exact recycle to the next matrix, then a refined solve from the recycled space
        solver.recycle(mats[1], 0)
        x2, st, stats = solver.solve(mats[1], torch.as_tensor(bs[1], device="cuda"))
        assert st == 0 and stats["converged"] == 1, stats
        assert_true_residual(As[1], bs[1], x2.cpu().numpy(), rel_tol)
    finally:
        solver.close()
