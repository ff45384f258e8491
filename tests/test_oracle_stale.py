"""Pins of the oracle's rank rule for an installed SAU and of its failure
detection for the inexact variant (Section 3.6).

The rank rule is pinned by closed forms: for two columns at angle theta the
QR has |R_22| = ||c|| sin(theta).  The stale-SAU rule rests on the embedding
bound of Section 3 (Eq. (sketch)): with an exact SAU the true residual lies in
the embedded subspace, so res <= sres / (1 - eps).  The pins check that the
rule never fires on the exact variant, and that on the paper's Section 6.3
operator family the inexact variant fails on the third problem (its true
residual grows past ||b|| while it runs, as Section 6.3 reports) and the rule
turns it into a converging run."""
import numpy as np
import pytest

import workloads as W
from oracle import sdr as O
from oracle.sketch import SparseSign


def _two_columns(theta, s=200, scale=3.0):
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((s, 2)))
    a = scale * Q[:, 0]
    c = scale * (np.cos(theta) * Q[:, 0] + np.sin(theta) * Q[:, 1])
    return np.stack([a, c], axis=1)


def test_rank_rule_closed_forms():
    s = 200
    R = np.linalg.qr(_two_columns(1e-6), mode="r")
    assert abs(abs(R[1, 1]) - 3.0 * np.sin(1e-6)) < 1e-12  # |R_22| = ||c|| sin(theta)
    assert not O.sau_rank_deficient(_two_columns(1e-10))  # 3e-10 > s eps ||c|| = 1.3e-13
    assert O.sau_rank_deficient(_two_columns(3e-14))      # 9e-14 <= s eps ||c||, though above eps ||c||
    assert O.sau_rank_deficient(_two_columns(1e-16))      # below the threshold
    assert O.sau_rank_deficient(_two_columns(0.0))        # duplicated columns
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((s, 8)))
    assert not O.sau_rank_deficient(Q)                    # orthonormal: full rank
    Z = Q.copy()
    Z[:, 3] = 0.0
    assert O.sau_rank_deficient(Z)                        # a zero column
    Z = Q.copy()
    Z[7, 2] = np.nan
    assert O.sau_rank_deficient(Z)                        # not finite
    assert not O.sau_rank_deficient(np.zeros((s, 0)))     # an empty space is no error


def _cd_sequence(n):
    As = [W.make_cd_paper(n, a) for a in (0.0, 5.0, 20.0)]
    return As, [np.ones(As[0].n)] * 3


@pytest.mark.parametrize("n", [30])
def test_stale_rule_silent_on_exact_variant(n):
    As, bs = _cd_sequence(n)
    S = SparseSign(231114206, As[0].n, 200, 8)
    kw = dict(m=40, k=10, t=2, rel_tol=1e-6, exact=True, max_cycles=30)
    a = O.solve_sequence(As, bs, S, stale_check=False, **kw)
    b = O.solve_sequence(As, bs, S, stale_check=True, **kw)
    for p, q in zip(a, b):
        assert q.sau_refreshes == 0
        assert np.array_equal(p.x, q.x) and p.matvecs == q.matvecs
        for checks in p.checks:  # the embedding bound at every true-residual check
            for (_, sres, res) in checks:
                assert res <= O.STALE_RATIO * sres


def test_stale_rule_rescues_inexact_variant():
    As, bs = _cd_sequence(30)
    S = SparseSign(231114206, As[0].n, 200, 8)
    kw = dict(m=40, k=10, t=2, rel_tol=1e-6, max_cycles=30)
    exact = O.solve_sequence(As, bs, S, exact=True, **kw)
    plain = O.solve_sequence(As, bs, S, exact=False, **kw)
    checked = O.solve_sequence(As, bs, S, exact=False, stale_check=True, **kw)
    bn = np.linalg.norm(bs[2])
    # Section 6.3's finding: the inexact variant fails on the third problem,
    # its true residual growing past ||b|| while the sketched one falls
    assert not plain[2].converged and plain[2].res > bn
    # the rule fires, and every problem converges
    assert all(o.converged for o in checked)
    assert sum(o.sau_refreshes for o in checked) >= 1
    # at most a few cycles more than the exact variant
    assert sum(o.matvecs for o in checked) <= sum(o.matvecs for o in exact) + 2 * (40 + 1)
