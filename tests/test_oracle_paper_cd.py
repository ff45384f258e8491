"""The oracle on the paper's own sequence experiment (Section 6.3), with the
counts its table prints (tests/golden/cd_paper_section_6_3.json).

Three 2D convection-diffusion systems (n = 500, N = 250,000, convection
alpha = 0, 5, 20, b = ones), solved in sequence with m = 80 Arnoldi steps per
cycle and k = 20 recycled columns (Algorithm 1's meaning of m), t = 2, at most
10 restarts per system.  Readings: the target residual 1e-2 is taken relative
to ||b||.  The sketch is the paper's own, a subsampled randomised DCT with
s = 8 m_max = 640 (Section 6).  Pinned:
  * the inexact variant (S A^(i) U kept) converges on the first two problems
    and fails on the third, where its true residual grows past ||b|| although
    the sketched residuals keep falling; its total count of matrix-vector
    products is the printed 1,886 within 3 % (the third problem runs into the
    restart cap, so the total is fixed mainly by the first two);
  * the exact variant (S A^(i+1) U recomputed) converges on all three
    problems, with a count inside a loose band around the printed 1,971 (it
    comes out about 20 % lower, with this sketch and with the sparse sign).
About three and a half minutes on one core."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import sdr as osdr
from oracle.sketch import SubsampledDCT

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.slow
def test_section_6_3_exact_and_inexact_recycling():
    fx = json.load(open(os.path.join(HERE, "golden", "cd_paper_section_6_3.json")))
    n = fx["n"]
    N = n * n
    As = [W.make_cd_paper(n, a) for a in fx["alpha"]]
    b = np.ones(N)
    k = fx["k_augmentation"]
    m = fx["m_krylov_dimension"]
    S = SubsampledDCT(231114206, N, 8 * fx["m_krylov_dimension"])
    kw = dict(m=m, k=k, t=2, rel_tol=fx["target_residual"], max_cycles=10)

    try:  # numpy's BLAS threads only spin on these memory-bound vector operations
        from threadpoolctl import threadpool_limits
        limit = threadpool_limits(1)
    except ImportError:
        limit = None
    exact = osdr.solve_sequence(As, [b] * 3, S, exact=True, **kw)
    assert [r.converged for r in exact] == [True, True, True]
    mv = sum(r.matvecs for r in exact)
    paper = fx["table"]["gmres_sdr_exact"]["matvecs"]
    assert 0.6 * paper <= mv <= 1.4 * paper, mv

    # the inexact variant (Section 3.6: S A^(i) U kept); its first solve is the
    # exact variant's (nothing is carried into problem 1)
    inexact = [exact[0]]
    for A in As[1:]:
        prev = inexact[-1]
        inexact.append(osdr.solve(A, b, S, U=prev.U, SU=prev.SU, SAU=prev.SAU, **kw))
    if limit is not None:
        limit.unregister()
    fails = fx["inexact_fails_on_problem"] - 1
    assert [r.converged for r in inexact] == [i != fails for i in range(3)]
    assert inexact[fails].res > np.linalg.norm(b)
    mv = sum(r.matvecs for r in inexact)
    paper = fx["table"]["gmres_sdr_inexact"]["matvecs"]
    assert 0.97 * paper <= mv <= 1.03 * paper, mv
    # within each cycle of the failing solve the sketched residual does not increase
    for cyc in inexact[fails].sres_per_cycle:
        assert all(b_ <= a_ * (1 + 1e-12) for a_, b_ in zip(cyc, cyc[1:]))
