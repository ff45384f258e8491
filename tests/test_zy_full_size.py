"""Parity at the full size of the timed workload.

The 3D convection-diffusion sequence on a 128^3 grid (N = 2,097,152, 14.6 M
nonzeros) with m = 100, k = 20, t = 2, s = 480, zeta = 8, rel_tol 1e-8 and
exact recycling: the solver parameters, matrices, right-hand sides and launch
path (captured CUDA graphs) of the timed benchmark.

A whole solve at this size is out of the oracle's reach, so the checks are the
outputs it computes within seconds, and properties that hold at any size:
  * the sketched residuals of the first 12 Arnoldi steps of the first cycle
    against the oracle's first 12 steps of Algorithm 1 on the same system;
  * the true residual ||b - A x|| of every solve, recomputed on the host,
    below tol (up to the rounding of that recomputation);
  * after the exact recycle to the next matrix (Section 3.6), sampled columns
    of SAU against S (A_next u) formed by the oracle's matvec and sketch;
  * the next system's first 12 sketched residuals against the oracle's cycle
    started from the recycle space the GPU handed over.
This file runs near the end of the suite: it holds about 2 GB of device memory
for its handle.
"""
import numpy as np
import pytest

import bench
import workloads as W
from oracle import sdr as osdr
from oracle.sketch import SparseSign

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps
STEPS = 12


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


def abs_csr(A):
    return W.CSR(A.n, A.rowptr, A.col, np.abs(A.val))


def abs_sketch(S, v):
    """|S| v (every sign taken as +1)."""
    w = np.broadcast_to(v[:, None], S.rows.shape)
    return np.bincount(S.rows.ravel(), weights=w.ravel(), minlength=S.s) * S.scale


def assert_true_residual(A, b, x, tol_rel):
    """||b - A x|| <= tol ||b|| + the rounding of the two residual products (the
    GPU's, which decided convergence, and the host's: each at most 8 eps
    (|A| |x|) per row for rows of at most 7 entries)."""
    r = b - osdr.csr_matvec(A, x)
    slack = 16 * EPS * np.linalg.norm(osdr.csr_matvec(abs_csr(A), np.abs(x)))
    assert np.linalg.norm(r) <= tol_rel * np.linalg.norm(b) + slack


def assert_sres_close(gpu, ref, bnorm):
    """Per step: |gpu - ref| <= 1e-8 |ref| + 1e-13 ||b|| (the bar of the
    smaller parity cases)."""
    gpu, ref = np.asarray(gpu, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    bad = np.nonzero(np.abs(gpu - ref) > 1e-8 * np.abs(ref) + 1e-13 * bnorm)[0]
    assert bad.size == 0, f"steps {bad[:8]}: gpu {gpu[bad[:4]]} ref {ref[bad[:4]]}"


def test_full_size_sequence_steps_residuals_and_exact_recycle(P):
    cfg = bench.WORKLOAD
    A0, dvec, diag_pos = bench.make_inputs(cfg)
    N = A0.n
    assert N == 128 ** 3
    m, k, t, s, zeta, rel_tol = cfg["m"], cfg["k"], cfg["t"], cfg["s"], cfg["zeta"], cfg["rel_tol"]
    # system i of the timed sequence: A0 + i eps D, right-hand side i - 1
    As = [W.CSR(N, A0.rowptr, A0.col, bench.system_values(A0, dvec, diag_pos, i, cfg["eps"])) for i in (1, 2)]
    bs = [W.rhs(N, bench.replica_rhs_seed(0, i)) for i in (0, 1)]
    S = SparseSign(cfg["seed"], N, s, zeta)
    solver = P.Solver(N, m, k, t, s, zeta, cfg["seed"], rel_tol)
    try:
        # ---- system 1 from x0 = 0 and an empty recycle space
        Ad1 = P.CSRDevice.from_numpy(As[0])
        x1, st, stats = solver.solve(Ad1, dev(bs[0]))
        assert st == 0 and stats["converged"] == 1, stats
        sres1, _ = solver.history()
        bn1 = np.linalg.norm(bs[0])
        ref1 = osdr.cycle(As[0], bs[0], None, None, None, S, rel_tol * bn1, STEPS, t, k)
        assert_sres_close(sres1[:STEPS], ref1.sres[:STEPS], bn1)
        assert_true_residual(As[0], bs[0], x1.cpu().numpy(), rel_tol)
        del Ad1

        # ---- exact recycle to A^(2): SAU = S A^(2) U, sampled columns
        Ad2 = P.CSRDevice.from_numpy(As[1])
        solver.recycle(Ad2, 0)
        U, SU, SAU = P.sdr_recycle_export(solver.h, N, s)
        kd = U.shape[1]
        assert 1 <= kd <= k + 1
        Uh = U.cpu().numpy()
        SUh = np.ascontiguousarray(SU.cpu().numpy())
        SAUh = np.ascontiguousarray(SAU.cpu().numpy())
        for c in sorted({0, kd // 2, kd - 1}):
            u = np.ascontiguousarray(Uh[:, c])
            ref = S.apply(osdr.csr_matvec(As[1], u))
            # rounding: both products (8 eps |A| |u| per row, through |S|) and the
            # host's sums of about N zeta / s terms per sketch row
            bound = 64 * EPS * abs_sketch(S, osdr.csr_matvec(abs_csr(As[1]), np.abs(u))) \
                + 1e-11 * np.linalg.norm(ref)
            err = np.abs(SAUh[:, c] - ref)
            assert np.all(err <= bound), (c, float(err.max()), float(np.linalg.norm(ref)))

        # ---- system 2 from the recycled space
        x2, st, stats = solver.solve(Ad2, dev(bs[1]))
        assert st == 0 and stats["converged"] == 1, stats
        sres2, _ = solver.history()
        bn2 = np.linalg.norm(bs[1])
        ref2 = osdr.cycle(As[1], bs[1], np.ascontiguousarray(Uh), SUh, SAUh, S, rel_tol * bn2, STEPS, t, k)
        assert_sres_close(sres2[:STEPS], ref2.sres[:STEPS], bn2)
        assert_true_residual(As[1], bs[1], x2.cpu().numpy(), rel_tol)
    finally:
        solver.close()
