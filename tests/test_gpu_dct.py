"""The second sketch family on the GPU: the subsampled randomised DCT of the
paper's experiments (Section 6, S = sqrt(N/s) P F E), against the oracle's
SubsampledDCT with the same draws (workloads.dct_draws).

Bars: the sketch of random vectors within 1e-13 of ||S x|| (both sides sum in
FP64, in different orders); a solve's first-cycle sketched residuals within
1e-8 relative and its solution within 1e-6; the paper's Section 6.3 sequence
with this sketch at s = 480 and at the paper's own s = 640 against the
oracle's runs (tests/golden/paper_cd_dct_s480.json, paper_cd_dct_s640.json):
convergence, cycles within one, and the inexact variant's failure on the
third problem."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import sdr as osdr
from oracle.sketch import SubsampledDCT

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 231114206
GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2311_14206_gb300 as P
    return P


def dct_solver(P, n, m, k, s, tol=1e-8, **kw):
    solver = P.Solver(n, m, k, 2, s, 8, SEED, tol, sketch_kind=1, **kw)
    signs, rows = W.dct_draws(SEED, n, s)
    solver.set_sketch_draws(signs, rows)
    return solver


@pytest.mark.parametrize("n,s", [(5000, 120), (300001, 480), (777, 37)])
def test_dct_sketch_matches_oracle(P, n, s):
    solver = dct_solver(P, n, 10, 2, s)
    S = SubsampledDCT(SEED, n, s)
    rng = np.random.default_rng(n)
    for trial in range(2):
        x = rng.standard_normal(n) * (10.0 ** (3 * trial))
        y = P.sdr_sketch(solver.h, torch.as_tensor(x, device="cuda"), s).cpu().numpy()
        ref = S.apply(x)
        assert np.max(np.abs(y - ref)) <= 1e-13 * np.linalg.norm(ref), np.max(np.abs(y - ref))
    e = np.zeros(n)
    e[n // 2] = 1.0
    y = P.sdr_sketch(solver.h, torch.as_tensor(e, device="cuda"), s).cpu().numpy()
    assert np.allclose(y, S.apply(e), rtol=0, atol=1e-15)
    solver.close()


def test_dct_solve_cd2d_64_matches_oracle(P):
    A = W.make_cd2d(64, (10.0, 10.0))
    b = W.rhs(A.n)
    m, k, s, tol = 50, 10, 120, 1e-8
    solver = dct_solver(P, A.n, m, k, s, tol)
    x, st, stats = solver.solve(P.CSRDevice.from_numpy(A), torch.as_tensor(b, device="cuda"))
    sres, log = solver.history()
    solver.close()
    ref = osdr.solve(A, b, SubsampledDCT(SEED, A.n, s), m=m, k=k, t=2, rel_tol=tol)
    xh = x.cpu().numpy()
    bn = np.linalg.norm(b)
    assert st == 0 and ref.converged
    assert np.linalg.norm(b - osdr.csr_matvec(A, xh)) / bn <= tol * (1 + 1e-9)
    assert np.linalg.norm(xh - ref.x) / np.linalg.norm(ref.x) <= 1e-6
    assert abs(stats["cycles"] - ref.cycles) <= 1
    r0 = np.asarray(ref.sres_per_cycle[0])
    g0 = np.asarray(sres[:r0.size])
    assert np.all(np.abs(g0 - r0) <= 1e-8 * r0 + 1e-13 * bn)


def test_dct_handle_rejects_other_sizes_and_bad_draws(P):
    solver = P.Solver(1000, 10, 2, 2, 40, 8, SEED, 1e-8, sketch_kind=1)
    signs, rows = W.dct_draws(SEED, 900, 40)
    with pytest.raises(P.SdrError):  # a sign that is not +-1
        bad = signs.copy()
        bad[3] = 0
        solver.set_sketch_draws(bad, rows)
    with pytest.raises(P.SdrError):  # rows not increasing
        solver.set_sketch_draws(signs, rows[::-1].copy())
    solver.set_sketch_draws(signs, rows)
    A = W.make_cd2d(31)  # 961 rows: not the size the draws were set for
    with pytest.raises(P.SdrError):
        solver.solve(P.CSRDevice.from_numpy(A), torch.as_tensor(W.rhs(A.n), device="cuda"))
    solver.close()


@pytest.mark.parametrize("variant", ["exact", "inexact"])
@pytest.mark.parametrize("golden", ["paper_cd_dct_s480.json", "paper_cd_dct_s640.json"])
def test_section_6_3_with_the_papers_sketch(P, variant, golden):
    """s = 640 is the paper's own size (8 m_max, Section 6)."""
    gold = json.load(open(os.path.join(GOLDEN_DIR, golden)))
    p = gold["params"]
    ref = gold["variants"][variant]["problems"]
    As = [W.make_cd_paper(p["n"], a) for a in p["alpha"]]
    N = As[0].n
    b = np.ones(N)
    bn = np.linalg.norm(b)
    solver = dct_solver(P, N, p["m"], p["k"], p["s"], p["rel_tol"], max_cycles=p["max_cycles"])
    bd = torch.as_tensor(b, device="cuda")
    for i, (A, r) in enumerate(zip(As, ref)):
        Ad = P.CSRDevice.from_numpy(A)
        if i > 0:
            solver.recycle(Ad, 0 if variant == "exact" else 1)
        x, st, stats = solver.solve(Ad, bd)
        sres, _ = solver.history()
        true_rel = np.linalg.norm(b - osdr.csr_matvec(A, x.cpu().numpy())) / bn
        where = f"{variant} problem {i + 1}"
        assert bool(stats["converged"]) == r["converged"], (where, stats["final_rel_res"], r["rel_res"])
        assert abs(stats["cycles"] - r["cycles"]) <= 1, (where, stats["cycles"], r["cycles"])
        if r["converged"]:
            assert true_rel < p["rel_tol"], where
        else:
            assert true_rel > 1.0 and r["rel_res"] > 1.0, (where, true_rel)
        if i == 0:
            r0 = np.asarray(r["first_cycle_sres"])
            g0 = np.asarray(sres[:r0.size])
            assert np.all(np.abs(g0 - r0) <= 1e-8 * r0 + 1e-13 * bn), where
    solver.close()
