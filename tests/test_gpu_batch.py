"""The batched form: independent systems of uneven sizes, each with its own
handle, stream and recycle space, solved in lockstep by sdr_solve_batch with
every restart cycle replayed from a captured CUDA graph.

Bars: every system's solution within 1e-6 relative of the FP64 oracle's
sequence solve with the true residual below tol and the cycle count within
one; the batched solve agrees with the same handles solved one at a time with
direct launches (no graphs) to rounding (1e-9 relative).
"""
import numpy as np
import pytest

import workloads as W
from oracle import sdr as osdr
from oracle.sketch import SparseSign

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 231114206
M, K, T, S, ZETA, TOL = 40, 10, 2, 100, 8, 1e-8


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


def systems():
    """Four 2D systems of uneven sizes, convection drawn as in the batched workload."""
    rng = np.random.default_rng([W.SEEDS["grid"], 4])
    out = []
    for i, n in enumerate((24, 31, 40, 17)):
        conv = tuple(rng.uniform(1.0, 50.0, size=2))
        A0 = W.make_cd2d(n, conv)
        dvec = W.diag_perturbation(A0.n, tag=i)
        out.append((A0, dvec))
    return out


def test_batch_sequence_matches_oracle_and_single_solves(P):
    sysl = systems()
    nseq = 2
    handles = [P.Solver(A0.n, M, K, T, S, ZETA, SEED, TOL, stream=torch.cuda.Stream()) for A0, _ in sysl]
    singles = [P.Solver(A0.n, M, K, T, S, ZETA, SEED, TOL, graphs=False) for A0, _ in sysl]
    refs = []
    for (A0, dvec) in sysl:
        As = list(W.sequence_matrices(A0, nseq, 1e-3 * 100, dvec))
        bs = [W.rhs(A0.n, 100 + i) for i in range(nseq)]
        refs.append((As, bs, osdr.solve_sequence(As, bs, SparseSign(SEED, A0.n, S, ZETA), m=M, k=K, t=T,
                                                 rel_tol=TOL)))
    for step in range(nseq):
        mats = [P.CSRDevice.from_numpy(r[0][step]) for r in refs]
        bsd = [dev(r[1][step]) for r in refs]
        xs = [torch.zeros_like(b) for b in bsd]
        if step > 0:
            P.sdr_recycle_batch([h.h for h in handles], mats, 0)
        torch.cuda.synchronize()
        st, stats = P.sdr_solve_batch([h.h for h in handles], mats, bsd, xs)
        torch.cuda.synchronize()
        assert st == 0
        for i, (r, x, stt) in enumerate(zip(refs, xs, stats)):
            A, b, ref = r[0][step], r[1][step], r[2][step]
            xh = x.cpu().numpy()
            bn = np.linalg.norm(b)
            assert stt["converged"] == 1
            assert np.linalg.norm(b - osdr.csr_matvec(A, xh)) / bn <= TOL * (1 + 1e-9)
            assert np.linalg.norm(xh - ref.x) / np.linalg.norm(ref.x) <= 1e-6
            assert abs(stt["cycles"] - ref.cycles) <= 1
            # the same system on a handle of its own, direct launches
            if step > 0:
                singles[i].recycle(mats[i], 0)
            xs1, st1, stats1 = singles[i].solve(mats[i], bsd[i])
            assert st1 == 0 and stats1["cycles"] == stt["cycles"]
            assert np.linalg.norm(xs1.cpu().numpy() - xh) / np.linalg.norm(xh) <= 1e-9
    for h in handles + singles:
        h.close()


def test_batch_rejects_bad_arguments(P):
    A0, _ = systems()[0]
    h = P.Solver(A0.n, M, K, T, S, ZETA, SEED, TOL)
    A = P.CSRDevice.from_numpy(A0)
    b = dev(W.rhs(A0.n))
    with pytest.raises(P.SdrError):  # the same handle twice
        P.sdr_solve_batch([h.h, h.h], [A, A], [b, b], [torch.zeros_like(b), torch.zeros_like(b)])
    st, stats = P.sdr_solve_batch([], [], [], [])
    assert st == 0 and stats == []
    h.close()
