"""Error paths of the C ABI on the GPU, each made on the host (no GPU fault):
a lucky breakdown that converges, a NaN or an Inf in the inputs, an exact
breakdown that does not converge, a singular matrix that stalls, and a
rank-deficient recycle space.  After each, the same handle must solve an
ordinary system exactly as the oracle does."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import sdr as osdr
from oracle.sketch import SparseSign

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 231114206
M, K, T, S, ZETA, TOL = 20, 4, 2, 60, 8, 1e-8


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


def diag_csr(d):
    n = d.size
    return W.stencils.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
                          np.asarray(d, dtype=np.float64))


def ordinary_solve_matches_oracle(P, solver, n_side=24, max_cycles=200):
    """The handle, after an error, still solves a 2D convection-diffusion system
    as the oracle does (its recycle space dropped first: another matrix), with
    the handle's cycle cap."""
    A = W.make_cd2d(n_side)
    b = W.rhs(A.n, 3)
    solver.recycle(None, 2)
    x, st, stats = solver.solve(P.CSRDevice.from_numpy(A), dev(b))
    ref = osdr.solve(A, b, SparseSign(SEED, A.n, S, ZETA), m=M, k=K, t=T, rel_tol=TOL, max_cycles=max_cycles)
    xh = x.cpu().numpy()
    assert st == (0 if ref.converged else 4) and stats["converged"] == int(ref.converged)
    assert np.linalg.norm(xh - ref.x) / np.linalg.norm(ref.x) <= 1e-6
    assert abs(stats["cycles"] - ref.cycles) <= 1


def test_lucky_breakdown_converges(P):
    """A = 2I, b = e_3: H(2,1) = 0 after one step; the forced check finds the
    exact solution b/2 (the oracle's pin of the same case)."""
    n = 600
    A = diag_csr(np.full(n, 2.0))
    b = np.zeros(n)
    b[3] = 1.0
    ref = osdr.solve(A, b, SparseSign(SEED, n, S, ZETA), m=M, k=K, t=T, rel_tol=TOL)
    assert ref.converged and ref.cycles == 1 and np.allclose(ref.x, b / 2, rtol=0, atol=1e-15)
    solver = P.Solver(n, M, K, T, S, ZETA, SEED, TOL)
    x, st, stats = solver.solve(P.CSRDevice.from_numpy(A), dev(b))
    xh = x.cpu().numpy()
    assert st == 0 and stats["converged"] == 1 and stats["cycles"] == 1
    assert np.abs(xh - ref.x).max() <= 1e-15
    _, log = solver.history()
    assert log[0]["steps"] == 1 and (log[0]["flags"] & 2)  # one column, breakdown flagged
    ordinary_solve_matches_oracle(P, solver)
    solver.close()


@pytest.mark.parametrize("where", ["b", "A", "x0"])
@pytest.mark.parametrize("bad", [math.nan, math.inf])
def test_nonfinite_input_is_breakdown(P, where, bad):
    A = W.make_cd2d(24)
    b = W.rhs(A.n)
    x0 = np.zeros(A.n)
    if where == "b":
        b = b.copy()
        b[17] = bad
    elif where == "A":
        A = A.copy()
        A.val[40] = bad
    else:
        x0[5] = bad
    solver = P.Solver(A.n, M, K, T, S, ZETA, SEED, TOL)
    xd = dev(x0)
    st, stats = P.sdr_solve(solver.h, P.CSRDevice.from_numpy(A), dev(b), xd, allow=(5,))
    assert st == 5  # SDR_ERR_BREAKDOWN
    assert stats["cycles"] == 0  # caught before any cycle
    assert np.array_equal(xd.cpu().numpy(), x0, equal_nan=True)  # x unchanged
    ordinary_solve_matches_oracle(P, solver)
    solver.close()


def test_exact_breakdown_without_convergence(P):
    """Row and column i of A zero, b = e_i: A v_1 = 0, so H(1,1) = H(2,1) = 0
    and SAW's only column is zero.  The forced check leaves x unchanged
    (a zero pivot of R contributes nothing to y) and res = ||b|| >= tol:
    SDR_ERR_BREAKDOWN after one cycle."""
    A = W.make_cd2d(20)
    i = 123
    A = A.copy()
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    A.val[(rows == i) | (A.col == i)] = 0.0
    b = np.zeros(A.n)
    b[i] = 1.0
    solver = P.Solver(A.n, M, K, T, S, ZETA, SEED, TOL)
    xd = dev(np.zeros(A.n))
    st, stats = P.sdr_solve(solver.h, P.CSRDevice.from_numpy(A), dev(b), xd, allow=(5,))
    assert st == 5 and stats["cycles"] == 1 and stats["converged"] == 0
    assert np.array_equal(xd.cpu().numpy(), np.zeros(A.n))
    assert abs(stats["final_res"] - 1.0) <= 1e-14
    ordinary_solve_matches_oracle(P, solver, n_side=20)
    solver.close()


def test_zero_row_stalls_not_converged(P):
    """A zero row i (its column kept) makes A singular with b_i out of reach:
    the residual cannot drop below |b_i|; max_cycles ends the solve with
    SDR_ERR_NOT_CONVERGED and a finite iterate."""
    A = W.make_cd2d(20).copy()
    i = 77
    A.val[A.rowptr[i]:A.rowptr[i + 1]] = 0.0
    b = W.rhs(A.n)
    solver = P.Solver(A.n, M, K, T, S, ZETA, SEED, TOL, max_cycles=3)
    xd = dev(np.zeros(A.n))
    st, stats = P.sdr_solve(solver.h, P.CSRDevice.from_numpy(A), dev(b), xd)
    xh = xd.cpu().numpy()
    assert st == 4 and stats["cycles"] == 3
    assert np.all(np.isfinite(xh))
    assert np.linalg.norm(b - osdr.csr_matvec(A, xh)) >= abs(b[i]) * (1 - 1e-12)
    ordinary_solve_matches_oracle(P, solver, n_side=20, max_cycles=3)
    solver.close()


def test_rank_deficient_recycle_space(P):
    """U imported with two equal columns: SAU = S A U has rank kd - 1, so
    Algorithm 1's R^{-1} does not exist.  sdr_recycle_import returns
    SDR_ERR_RANK (the oracle's rule says deficient) and drops the space; the
    same holds for sdr_recycle in exact mode on such a space."""
    A = W.make_cd2d(24)
    rng = np.random.default_rng(2)
    U = rng.standard_normal((A.n, 3))
    U[:, 2] = U[:, 0]
    SAU = SparseSign(SEED, A.n, S, ZETA).apply_cols(osdr.csr_matmat(A, U))
    assert osdr.sau_rank_deficient(SAU)
    assert not osdr.sau_rank_deficient(SAU[:, :2])
    solver = P.Solver(A.n, M, K, T, S, ZETA, SEED, TOL)
    Ad = P.CSRDevice.from_numpy(A)
    with pytest.raises(P.SdrError) as e:
        P.sdr_recycle_import(solver.h, Ad, dev(U))
    assert e.value.status == 6  # SDR_ERR_RANK
    assert P.sdr_recycle_dim(solver.h) == 0
    # exact recycling recomputes SAU = S A U: a rank-deficient U installed with a
    # full-rank (made-up) SU and SAU passes the import, then fails in sdr_recycle
    Sfake = np.random.default_rng(3).standard_normal((S, 3))
    P.sdr_recycle_import(solver.h, Ad, dev(U), dev(Sfake), dev(Sfake))
    assert P.sdr_recycle_dim(solver.h) == 3
    with pytest.raises(P.SdrError) as e:
        solver.recycle(Ad, 0)
    assert e.value.status == 6 and P.sdr_recycle_dim(solver.h) == 0
    # a full-rank space is accepted and used
    P.sdr_recycle_import(solver.h, Ad, dev(U[:, :2]))
    assert P.sdr_recycle_dim(solver.h) == 2
    ordinary_solve_matches_oracle(P, solver)
    solver.close()
