"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: sketch indices bit-exact; per-step sketched residuals within 1e-8
relative (floor 1e-13 ||b|| for rounding cancellation, the sres being formed
from O(||S b||) terms); final solutions within 1e-6 relative with the true
residual below tol; recycle spaces compared by principal angles.
"""
import numpy as np
import pytest

import workloads as W
from oracle import sdr as osdr
from oracle.sketch import SparseSign, sketch_indices

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


def saw_conditioning(cyc):
    """kappa(SAW) after each step of an oracle cycle recorded with record=True."""
    SAU, SAV = cyc.info["SAU_in"], cyc.info["SAV"]
    return np.array([np.linalg.cond(np.hstack([SAU, SAV[:, :j + 1]])) for j in range(SAV.shape[1])])


def sres_close(gpu, ref, bnorm, rel=1e-8, floor=1e-13, kappa=None):
    """|gpu - ref| <= rel |ref| + (floor + 64 eps kappa_j) ||b||.  The kappa term
    is the first-order sensitivity of a least-squares residual to rounding in
    SAW; it is negligible while eps kappa(SAW) << 1e-10 (all t = 2 workloads)."""
    gpu, ref = np.asarray(gpu), np.asarray(ref)
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    err = np.abs(gpu - ref)
    kap = np.zeros_like(ref) if kappa is None else np.asarray(kappa)[:ref.size]
    bound = rel * np.abs(ref) + (floor + 64 * np.finfo(float).eps * kap) * bnorm
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, f"steps {bad[:8]}: gpu {gpu[bad[:4]]} ref {ref[bad[:4]]}"
    return float(np.max(err / (np.abs(ref) + floor * bnorm)))


def principal_angle(X, Y):
    Qx, _ = np.linalg.qr(X)
    Qy, _ = np.linalg.qr(Y)
    sv = np.linalg.svd(Qx.T @ Qy, compute_uv=False)
    return float(np.arccos(np.clip(sv.min(), -1, 1)))


# ---------------------------------------------------------------- sketch
@pytest.mark.parametrize("n,s,zeta", [(5000, 120, 8), (4096, 480, 8), (3000, 37, 3), (2500, 100, 1), (6000, 768, 8),
                                      (4500, 640, 8)])
def test_sketch_columns_bit_exact(P, n, s, zeta):
    solver = P.Solver(n, m=10, k=2, t=2, s=s, zeta=zeta, seed=SEED)
    rng = np.random.default_rng(0)
    cols = sorted(set([0, 1, 2047, 2048, 2049, n - 1] + list(rng.integers(0, n, 40))))
    rows, signs = sketch_indices(SEED, s, zeta, np.array(cols))
    for i, c in enumerate(cols):
        e = torch.zeros(n, dtype=torch.float64, device="cuda")
        e[c] = 1.0
        y = P.sdr_sketch(solver.h, e, s).cpu().numpy()
        ref = np.zeros(s)
        ref[rows[i]] = signs[i] / np.sqrt(float(zeta))
        assert np.array_equal(y, ref), f"column {c}"
    solver.close()


@pytest.mark.parametrize("n", [5000, 2**21 + 123])
def test_sketch_random_vector(P, n):
    s, zeta = 480, 8
    solver = P.Solver(n, m=10, k=2, t=2, s=s, zeta=zeta, seed=SEED)
    x = np.random.default_rng(1).standard_normal(n)
    y = P.sdr_sketch(solver.h, dev(x), s).cpu().numpy()
    ref = SparseSign(SEED, n, s, zeta).apply(x)
    assert np.max(np.abs(y - ref)) <= 1e-13 * np.linalg.norm(ref)
    # bit-for-bit reproducible
    y2 = P.sdr_sketch(solver.h, dev(x), s).cpu().numpy()
    assert np.array_equal(y, y2)
    solver.close()


# ---------------------------------------------------------------- solves
def run_pair(P, A, b, m, k, t, s, zeta, tol, max_cycles=200, **kw):
    solver = P.Solver(A.n, m, k, t, s, zeta, SEED, tol, max_cycles=max_cycles, **kw)
    Ad = P.CSRDevice.from_numpy(A)
    x, st, stats = solver.solve(Ad, dev(b))
    sres, log = solver.history()
    ref = osdr.solve(A, b, SparseSign(SEED, A.n, s, zeta), m=m, k=k, t=t, rel_tol=tol, max_cycles=max_cycles,
                     record=True)
    return solver, Ad, x.cpu().numpy(), st, stats, sres, log, ref


def test_cd2d_64_first_cycle_and_solution(P):
    A = W.make_cd2d(64, (10.0, 10.0))
    b = W.rhs(A.n)
    m, k, t, s, zeta, tol = 50, 10, 2, 120, 8, 1e-8
    solver, Ad, x, st, stats, sres, log, ref = run_pair(P, A, b, m, k, t, s, zeta, tol)
    bn = np.linalg.norm(b)
    sres_close(sres[:len(ref.sres_per_cycle[0])], ref.sres_per_cycle[0], bn)
    assert st == 0 and stats["converged"] == 1
    assert abs(stats["cycles"] - ref.cycles) <= 1
    relres = np.linalg.norm(b - osdr.csr_matvec(A, x)) / bn
    assert relres <= tol * (1 + 1e-9)
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-6
    # second cycle (strict in free-running mode)
    n0 = len(ref.sres_per_cycle[0])
    sres_close(sres[n0:n0 + len(ref.sres_per_cycle[1])], ref.sres_per_cycle[1], bn)
    solver.close()


def test_cd2d_64_cycle_replay(P):
    """Each GPU cycle starts from the oracle's state at that cycle's start."""
    A = W.make_cd2d(64, (10.0, 10.0))
    b = W.rhs(A.n)
    m, k, t, s, zeta, tol = 50, 10, 2, 120, 8, 1e-8
    S = SparseSign(SEED, A.n, s, zeta)
    states = []
    ref = osdr.solve(A, b, S, m=m, k=k, t=t, rel_tol=tol, record=True,
                     cycle_hook=lambda c, x, r, U, SU, SAU, sf: states.append((x.copy(), U, SU, SAU)))
    Ad = P.CSRDevice.from_numpy(A)
    bn = np.linalg.norm(b)
    for ci, (x0, U, SU, SAU) in enumerate(states):
        solver = P.Solver(A.n, m, k, t, s, zeta, SEED, tol, max_cycles=1)
        if U is not None and U.shape[1]:
            P.sdr_recycle_import(solver.h, Ad, dev(U), dev(SU), dev(SAU))
        xd = dev(x0)
        st, stats = P.sdr_solve(solver.h, Ad, dev(b), xd)
        sres, log = solver.history()
        sres_close(sres, ref.sres_per_cycle[ci], bn)
        c = ref.cycle_log[ci]
        assert log[0]["checks"] == len(c.checks)
        assert abs(log[0]["res"] - c.res) <= 1e-8 * c.res + 1e-13 * bn
        # recycle space after the cycle: same span as the oracle's
        Ug, _, _ = P.sdr_recycle_export(solver.h, A.n, s)
        assert Ug.shape[1] == c.U.shape[1]
        assert principal_angle(Ug.cpu().numpy(), c.U) < 1e-6
        solver.close()


@pytest.mark.parametrize("t,k,zeta,s", [(1, 10, 8, 120), (3, 10, 8, 120), (4, 5, 4, 90), (2, 0, 8, 100),
                                        (2, 10, 1, 120), (2, 10, 8, 62), (2, 10, 8, 640), (2, 10, 8, 768)])
def test_parameter_edges_first_cycles(P, t, k, zeta, s):
    A = W.make_cd2d(40, (20.0, 5.0))  # N = 1600
    b = W.rhs(A.n, 7)
    m, tol = 50, 1e-8
    solver, Ad, x, st, stats, sres, log, ref = run_pair(P, A, b, m, k, t, s, zeta, tol, max_cycles=2)
    bn = np.linalg.norm(b)
    n0 = len(ref.sres_per_cycle[0])
    sres_close(sres[:n0], ref.sres_per_cycle[0], bn, kappa=saw_conditioning(ref.cycle_log[0]))
    if t == 2:  # the well-conditioned workloads keep the strict bar with no kappa term
        sres_close(sres[:n0], ref.sres_per_cycle[0], bn)
    if len(ref.sres_per_cycle) > 1 and len(log) > 1:
        sres_close(sres[n0:n0 + len(ref.sres_per_cycle[1])], ref.sres_per_cycle[1], bn,
                   kappa=saw_conditioning(ref.cycle_log[1]))
    solver.close()


def test_ragged_sizes_and_3d(P):
    A = W.make_cd3d(17, (20.0, 10.0, 5.0))  # N = 4913: two full sketch tiles and a ragged one
    b = W.rhs(A.n, 3)
    m, k, t, s, zeta, tol = 40, 8, 2, 120, 8, 1e-8
    solver, Ad, x, st, stats, sres, log, ref = run_pair(P, A, b, m, k, t, s, zeta, tol)
    bn = np.linalg.norm(b)
    sres_close(sres[:len(ref.sres_per_cycle[0])], ref.sres_per_cycle[0], bn)
    assert st == 0
    assert np.linalg.norm(b - osdr.csr_matvec(A, x)) / bn <= tol * (1 + 1e-9)
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-6
    solver.close()


def test_force_svd_path_same_span(P):
    """The truncated-SVD path and the full-rank path give the same recycle span."""
    A = W.make_cd2d(40, (10.0, 10.0))
    b = W.rhs(A.n, 2)
    m, k, t, s, zeta, tol = 40, 8, 2, 100, 8, 1e-8
    Ad = P.CSRDevice.from_numpy(A)
    out = []
    for force in (False, True):
        solver = P.Solver(A.n, m, k, t, s, zeta, SEED, tol, max_cycles=1, force_svd=force)
        x, st, stats = solver.solve(Ad, dev(b))
        sres, log = solver.history()
        assert (log[0]["flags"] & 1) == (1 if force else 0)
        U, _, _ = P.sdr_recycle_export(solver.h, A.n, s)
        out.append(U.cpu().numpy())
        solver.close()
    ref = osdr.solve(A, b, SparseSign(SEED, A.n, s, zeta), m=m, k=k, t=t, rel_tol=tol, max_cycles=1)
    assert principal_angle(out[0], out[1]) < 1e-7
    assert principal_angle(out[1], ref.U) < 1e-6


def test_sequence_exact_recycling(P):
    A0 = W.make_cd3d(16, (20.0, 10.0, 5.0))
    dvec = W.diag_perturbation(A0.n)
    As = list(W.sequence_matrices(A0, 3, 1e-3 * 1000, dvec))
    bs = [W.rhs(A0.n, i) for i in range(3)]
    m, k, t, s, zeta, tol = 40, 8, 2, 120, 8, 1e-8
    refs = osdr.solve_sequence(As, bs, SparseSign(SEED, A0.n, s, zeta), m=m, k=k, t=t, rel_tol=tol)
    solver = P.Solver(A0.n, m, k, t, s, zeta, SEED, tol)
    for i, (A, b, ref) in enumerate(zip(As, bs, refs)):
        Ad = P.CSRDevice.from_numpy(A)
        if i > 0:
            solver.recycle(Ad, 0)
        x, st, stats = solver.solve(Ad, dev(b))
        sres, log = solver.history()
        bn = np.linalg.norm(b)
        xh = x.cpu().numpy()
        assert st == 0
        assert np.linalg.norm(b - osdr.csr_matvec(A, xh)) / bn <= tol * (1 + 1e-9)
        assert np.linalg.norm(xh - ref.x) / np.linalg.norm(ref.x) <= 1e-6
        assert abs(stats["cycles"] - ref.cycles) <= 1
        sres_close(sres[:len(ref.sres_per_cycle[0])], ref.sres_per_cycle[0], bn)
    solver.close()


def test_already_converged_and_errors(P):
    A = W.make_cd2d(24)
    b = W.rhs(A.n)
    xs = np.linalg.solve(W.csr_to_dense(A), b)
    solver = P.Solver(A.n, 20, 4, 2, 40, 8, SEED, 1e-8)
    Ad = P.CSRDevice.from_numpy(A)
    xd = dev(xs)
    st, stats = P.sdr_solve(solver.h, Ad, dev(b), xd)
    assert st == 0 and stats["cycles"] == 0
    # size beyond n_max is rejected on the host
    big = P.CSRDevice.from_numpy(W.make_cd2d(30))
    with pytest.raises(P.SdrError):
        P.sdr_solve(solver.h, big, dev(W.rhs(900)), dev(np.zeros(900)))
    solver.close()
    with pytest.raises(P.SdrError):
        P.Solver(100, 20, 4, 2, 20, 8, SEED, 1e-8)  # s < m + k + 2


def irregular_matrix():
    """cd2d 64 x 64 with extra weak couplings: row 100 gets 300 more entries
    (longer than the integer SpMV's exact 64-bit row sums: summed in FP64),
    and rows 600 .. 1099 six more each, so that the second 512-row block holds
    more entries than one shared-memory stage (read from global memory
    instead).  Entries of 1e-3 and a diagonal raised by their sum keep the
    matrix as well conditioned as the stencil's."""
    import scipy.sparse as sp
    A0 = W.make_cd2d(64, (10.0, 10.0))
    n = A0.n
    M = sp.csr_matrix((A0.val, A0.col, A0.rowptr), shape=(n, n)).tolil()
    rng = np.random.default_rng(5)
    extra = [(100, c) for c in rng.choice(n, 300, replace=False)]
    for r in range(600, 1100):
        extra += [(r, c) for c in rng.choice(n, 6, replace=False)]
    for r, c in extra:
        if r != c:
            M[r, c] = M[r, c] + 1e-3 * (1 if rng.random() < 0.5 else -1)
            M[r, r] = M[r, r] + 1e-3
    M = M.tocsr()
    M.sort_indices()
    return W.stencils.CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64))


def test_irregular_rows_and_stage_overflow(P):
    A = irregular_matrix()
    lens = np.diff(A.rowptr)
    assert lens.max() > 252 and A.rowptr[1024] - A.rowptr[512] > 4096
    b = W.rhs(A.n, 4)
    m, k, t, s, zeta, tol = 50, 10, 2, 120, 8, 1e-8
    solver, Ad, x, st, stats, sres, log, ref = run_pair(P, A, b, m, k, t, s, zeta, tol)
    bn = np.linalg.norm(b)
    sres_close(sres[:len(ref.sres_per_cycle[0])], ref.sres_per_cycle[0], bn)
    assert st == 0 and stats["converged"] == 1
    assert abs(stats["cycles"] - ref.cycles) <= 1
    assert np.linalg.norm(b - osdr.csr_matvec(A, x)) / bn <= tol * (1 + 1e-9)
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-6
    solver.close()


def test_repeat_solves_bit_identical(P):
    """Every reduction of the FP64 path has a fixed order (the staged SpMV sums
    its dots per tile, whichever CTA took the tile), so repeated solves, with
    captured graphs or direct launches, give the same bits."""
    A = W.make_cd3d(24, (20.0, 10.0, 5.0))  # 13,824 rows: 14 tiles on up to 152 CTAs
    b = dev(W.rhs(A.n, 9))
    Ad = P.CSRDevice.from_numpy(A)
    outs = []
    for graphs in (True, True, False):
        solver = P.Solver(A.n, 40, 8, 2, 120, 8, SEED, 1e-10, graphs=graphs)
        x, st, stats = solver.solve(Ad, b)
        sres, _ = solver.history()
        outs.append((x.cpu().numpy(), stats["cycles"], np.asarray(sres)))
        assert st == 0
        solver.close()
    for x, cyc, sres in outs[1:]:
        assert cyc == outs[0][1]
        assert np.array_equal(sres, outs[0][2])
        assert np.array_equal(x, outs[0][0])


def test_trace_entries(P):
    """sdr_trace keeps one entry per profiled launch: on the stream it was
    issued to, ordered within each stream, end after start, and as many per
    class as sdr_profile_get counts; a cap bounds the list."""
    A = W.make_cd2d(40, (20.0, 5.0))
    b = dev(W.rhs(A.n, 2))
    Ad = P.CSRDevice.from_numpy(A)
    solver = P.Solver(A.n, 40, 8, 2, 120, 8, SEED, 1e-8)
    P.sdr_profile(solver.h, True)
    P.sdr_trace(solver.h, 1 << 16)
    x, st, stats = solver.solve(Ad, b)
    assert st == 0
    tr = P.sdr_trace_get(solver.h)
    prof = P.sdr_profile_get(solver.h)
    assert len(tr) == sum(n for n, _ in prof.values()) > 0
    for cls, (n, _) in prof.items():
        assert sum(1 for e in tr if e[0] == cls) == n
    assert all(e[1] in (0, 1) and 0.0 <= e[2] <= e[3] for e in tr)
    assert {e[1] for e in tr if e[0] == "spmv_dots"} == {0}
    assert {e[1] for e in tr if e[0] == "step_dense"} == {1}
    for s_ in (0, 1):
        starts = [e[2] for e in tr if e[1] == s_]
        assert starts == sorted(starts)
    P.sdr_trace(solver.h, 5)
    solver.solve(Ad, b)
    assert len(P.sdr_trace_get(solver.h)) == 5
    P.sdr_trace(solver.h, 0)
    assert P.sdr_trace_get(solver.h) == []
    P.sdr_profile(solver.h, False)
    solver.close()


# ------------------------------------------------- recycle product on tensor cores
@pytest.mark.parametrize("side,m,k,s,tol,maxc", [(17, 40, 10, 120, 1e-10, 200), (20, 128, 31, 200, 1e-15, 3),
                                                 (24, 60, 20, 200, 1e-10, 200)])
def test_recycle_product_tensor_cores_bit_identical(P, side, m, k, s, tol, maxc):
    """The recycle product U_new = [U V] P on the tcgen05 tensor cores (exact
    integer digit products) equals the integer-pipe product bit for bit, so the
    whole solve is bit-identical; sizes cover a ragged last tile (17^3 rows,
    odd), the widest SAW (d = kh + m = 32 + 128 = 160 columns: three full
    cycles of 128 steps toward an unreachable tolerance) and several cycles of
    recycling.  The solve also matches the oracle."""
    A = W.make_cd3d(side, (20.0, 10.0, 5.0))
    b = W.rhs(A.n, 11)
    out = []
    for integer in (False, True):
        solver = P.Solver(A.n, m, k, 2, s, 8, SEED, tol, max_cycles=maxc, integer_recycle=integer)
        x, st, stats = solver.solve(P.CSRDevice.from_numpy(A), dev(b))
        sres, log = solver.history()
        U, SU, SAU = P.sdr_recycle_export(solver.h, A.n, s)
        out.append((x.cpu().numpy(), st, stats, np.array(sres), U.cpu().numpy()))
        solver.close()
    (x0, st0, s0, h0, U0), (x1, st1, s1, h1, U1) = out
    assert st0 == st1 and s0["cycles"] >= 2 and s0["cycles"] == s1["cycles"]
    assert np.array_equal(U0, U1)
    assert np.array_equal(x0, x1) and np.array_equal(h0, h1)
    ref = osdr.solve(A, b, SparseSign(SEED, A.n, s, 8), m=m, k=k, t=2, rel_tol=tol, max_cycles=maxc)
    assert np.linalg.norm(x0 - ref.x) / np.linalg.norm(ref.x) <= 1e-6
    assert abs(s0["cycles"] - ref.cycles) <= 1


# ------------------------------------------------------- Givens-sine estimator
def test_givens_sines_match_oracle(P):
    """Per-step Givens sines and cosines of the GPU's cycles (read off its QR of
    SAW) against the oracle's Section 5 construction (QR of [SAU, SV], G, Givens
    rotations) for the first two cycles of the 64 x 64 workload; the second
    cycle is augmented (k recycled columns).  Bars: |ds| <= 1e-8 s + 1e-12 and
    |dc| <= 1e-7 c + 1e-10 (c = sqrt(1 - s^2) amplifies the error of s when s
    is close to one)."""
    from oracle import givens as G
    A = W.make_cd2d(64, (10.0, 10.0))
    b = W.rhs(A.n)
    m, k, t, s, zeta, tol = 50, 10, 2, 120, 8, 1e-8
    solver = P.Solver(A.n, m, k, t, s, zeta, SEED, tol)
    x, st, stats = solver.solve(P.CSRDevice.from_numpy(A), dev(b))
    sines, cosines = P.sdr_get_givens(solver.h)
    sres, log = solver.history()
    solver.close()
    assert len(sines) == len(sres)
    ref = osdr.solve(A, b, SparseSign(SEED, A.n, s, zeta), m=m, k=k, t=t, rel_tol=tol, record=True)
    off = 0
    for cyc, g in zip(ref.cycle_log[:2], log[:2]):
        info = cyc.info
        rs, rc, rsres = G.givens_sines(info["SAU_in"], info["SV"], info["H"], info["beta"])
        n = min(len(rs), g["steps"])
        gs, gc = np.asarray(sines[off:off + n]), np.asarray(cosines[off:off + n])
        assert np.all(np.abs(gs - rs[:n]) <= 1e-8 * rs[:n] + 1e-12), (off, np.max(np.abs(gs - rs[:n])))
        assert np.all(np.abs(gc - rc[:n]) <= 1e-7 * rc[:n] + 1e-10), (off, np.max(np.abs(gc - rc[:n])))
        # the Theorem's recurrence on the GPU's own numbers
        prev = np.concatenate([[gs[0] and sres[off] / gs[0]], sres[off:off + n - 1]])
        assert np.allclose(np.asarray(sres[off:off + n]), gs * prev, rtol=1e-12)
        off += g["steps"]
