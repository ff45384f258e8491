"""Pins of the oracle's building blocks, each against something other than the
oracle: a library routine that solves the same problem, a closed form, or an
invariant of the definition (CPU only).

  back_substitute       -- scipy's triangular solver
  sketched_ls           -- numpy's least-squares solver (Algorithm 1, QR-based
                           least squares)
  numerical_rank        -- spectra and matrices of known rank (Section 3.5)
  select_largest        -- ordering invariants, conjugate pairs kept whole
  invariant_basis       -- B Z = Z T with the selected eigenvalues as T's
  harmonic_ritz_update  -- exact harmonic Ritz values mu = 1/lambda when W
                           spans an invariant subspace of A, with any sketch
                           (Section 3.5)
  cycle                 -- a lucky breakdown (H(j+1, j) = 0) ends the cycle
                           with the exact solution; finite termination after
                           as many steps as the degree of the minimal
                           polynomial (Algorithm 1)
"""
import numpy as np
import pytest
import scipy.linalg

import oracle.sdr as ORACLE
import workloads as W
from oracle.sketch import SparseSign


def rng(i):
    return np.random.default_rng([2311, 14206, i])


def pin_back_substitute_matches_library_triangular_solve(O):
    g = rng(1)
    for n in (1, 2, 7, 40):
        R = np.triu(g.standard_normal((n, n))) + n * np.eye(n)
        z = g.standard_normal(n)
        y = O.back_substitute(R, z)
        ref = scipy.linalg.solve_triangular(R, z, lower=False)
        assert np.allclose(y, ref, rtol=1e-13, atol=1e-13)


def pin_sketched_ls_matches_library_least_squares(O):
    g = rng(2)
    for s, d in ((30, 1), (60, 12), (200, 45)):
        SAW = g.standard_normal((s, d))
        Sr0 = g.standard_normal(s)
        y, sres = O.sketched_ls(SAW, Sr0)
        ref, *_ = np.linalg.lstsq(SAW, Sr0, rcond=None)
        assert np.allclose(y, ref, rtol=1e-10, atol=1e-12)
        assert sres == pytest.approx(np.linalg.norm(Sr0 - SAW @ ref), rel=1e-10)
    # a right-hand side in the range of SAW is matched exactly
    SAW = g.standard_normal((40, 6))
    y0 = g.standard_normal(6)
    y, sres = O.sketched_ls(SAW, SAW @ y0)
    assert np.allclose(y, y0, rtol=1e-11) and sres < 1e-12 * np.linalg.norm(SAW @ y0)


def pin_numerical_rank_known_spectra_and_matrices(O):
    eps = np.finfo(np.float64).eps
    assert O.numerical_rank(np.array([]), 0) == 0
    assert O.numerical_rank(np.zeros(3), 3) == 0
    assert O.numerical_rank(np.ones(5), 5) == 5
    # threshold sigma_1 * d * eps: a value just above it counts, just below it does not
    d = 10
    assert O.numerical_rank(np.array([1.0, 1.01 * d * eps, 0.99 * d * eps]), d) == 2
    # matrices built with a known rank r (a gap of many orders of magnitude)
    g = rng(3)
    for s, d, r in ((80, 20, 7), (120, 30, 30), (60, 15, 1)):
        M = g.standard_normal((s, r)) @ g.standard_normal((r, d))
        sig = np.linalg.svd(M, compute_uv=False)
        assert O.numerical_rank(sig, d) == r


def pin_select_largest_invariants(O):
    g = rng(4)
    for trial in range(200):
        n = int(g.integers(1, 12))
        k = int(g.integers(0, n + 2))
        # real eigenvalues and conjugate pairs, with repeated moduli on purpose
        vals = []
        while len(vals) < n:
            if len(vals) + 2 <= n and g.random() < 0.4:
                a, b = g.integers(-3, 4), g.integers(1, 4)
                vals += [complex(a, b), complex(a, -b)]
            else:
                vals.append(complex(g.integers(-4, 5), 0))
        mu = np.array(vals)
        g.shuffle(mu)
        sel = O.select_largest(mu, k)
        kk = min(k, n)
        assert len(set(sel.tolist())) == len(sel)
        assert len(sel) in (kk, kk + 1)
        rest = np.setdiff1d(np.arange(n), sel)
        if len(sel) and len(rest):
            assert np.abs(mu[sel]).min() >= np.abs(mu[rest]).max()
        # a selected complex eigenvalue comes with its conjugate
        for i in sel:
            if mu[i].imag != 0:
                assert np.conj(mu[i]) in mu[sel]
        # one more than k only to keep a conjugate pair whole
        if len(sel) == kk + 1:
            a, b = mu[sel[-2]], mu[sel[-1]]
            assert a.imag != 0 and b == np.conj(a)
        # ties in modulus are broken by the larger real part
        for i in sel:
            for j in rest:
                if abs(mu[i]) == abs(mu[j]) and not (len(sel) == kk + 1 and i == sel[-1]):
                    assert mu[i].real >= mu[j].real


def pin_select_largest_real_distinct_matches_sort(O):
    g = rng(5)
    mu = g.standard_normal(15).astype(complex)
    for k in range(16):
        sel = O.select_largest(mu, k)
        assert list(sel) == list(np.argsort(-np.abs(mu), kind="stable")[:k])


def pin_invariant_basis_spans_an_invariant_subspace(O):
    g = rng(6)
    for n, k in ((6, 2), (12, 5), (20, 7)):
        B = g.standard_normal((n, n))
        mu, Y = np.linalg.eig(B)
        sel = O.select_largest(mu, k)
        Z = O.invariant_basis(mu, Y, sel)
        assert Z.dtype == np.float64 and Z.shape == (n, len(sel))
        assert np.allclose(Z.T @ Z, np.eye(len(sel)), atol=1e-12)
        T = Z.T @ B @ Z
        assert np.linalg.norm(B @ Z - Z @ T) < 1e-10 * np.linalg.norm(B)
        got = np.sort_complex(np.linalg.eigvals(T))
        assert np.allclose(got, np.sort_complex(mu[sel]), atol=1e-9)


def pin_harmonic_ritz_exact_on_an_invariant_subspace(O, with_sketch=False):
    """A = X diag(lambda) X^{-1}, W = X(:, :d): A W = W diag(lambda(:d)), so the
    pencil of Section 3.5 has the exact eigenvalues mu = 1/lambda_i with any
    subspace embedding, and P picks the k of smallest |lambda|."""
    g = rng(7 + with_sketch)
    n, d, k, s = 60, 12, 4, 40
    lam = np.concatenate([g.uniform(0.5, 5.0, d) * g.choice([-1, 1], d), g.uniform(6, 9, n - d)])
    X = g.standard_normal((n, n)) + 3 * np.eye(n)
    A = X @ np.diag(lam) @ np.linalg.inv(X)
    W = X[:, :d]
    if with_sketch:
        S = SparseSign(231114206, n, s, 4).dense()
    else:
        S = np.eye(n)
    P, info = O.harmonic_ritz_update(S @ A @ W, S @ W, k)
    assert info["ell"] == d
    assert np.allclose(np.sort(info["mu"].real), np.sort(1.0 / lam[:d]), rtol=1e-8)
    assert np.abs(info["mu"].imag).max() < 1e-8
    # the recycled directions W P span the eigenvectors of the k smallest |lambda|
    want = X[:, np.argsort(np.abs(lam[:d]))[:k]]
    Qa, _ = np.linalg.qr(W @ P)
    Qb, _ = np.linalg.qr(want)
    cosines = np.linalg.svd(Qa.T @ Qb, compute_uv=False)
    assert cosines.min() > 1 - 1e-8


def diag_csr(d):
    n = d.size
    return W.CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.asarray(d, dtype=np.float64))


def pin_lucky_breakdown_stops_the_cycle(O):
    """A = 2 I, b = e_3: A v_1 = 2 v_1 exactly, so H(2, 1) = 0 at the first step.
    The forced check finds x = b / 2.  With tol = 0 no sres can trigger a check,
    so only the breakdown rule ends the cycle after one column."""
    n = 16
    A = diag_csr(np.full(n, 2.0))
    b = np.zeros(n)
    b[3] = 1.0
    S = SparseSign(5, n, 12, 3)
    c = O.cycle(A, b, None, None, None, S, 1e-12, 8, 2, 2)
    assert c.converged and c.j == 1 and len(c.sres) == 1
    assert np.allclose(c.x_tilde, b / 2, rtol=0, atol=1e-15)
    c0 = O.cycle(A, b, None, None, None, S, 0.0, 8, 2, 2)
    assert not c0.converged and c0.j == 1 and len(c0.sres) == 1 and len(c0.checks) == 1


def pin_finite_termination(O):
    """A diagonal A with three distinct eigenvalues: the minimal polynomial of A
    with respect to a generic b has degree 3, so GMRES with full orthogonalisation
    over those steps (t = 3) reaches A^-1 b at the third step and not before."""
    g = rng(9)
    n = 30
    d = g.choice([2.0, 5.0, -3.0], n)
    d[:3] = [2.0, 5.0, -3.0]
    A = diag_csr(d)
    b = g.standard_normal(n)
    S = SparseSign(6, n, 20, 4)
    tol = 1e-10 * np.linalg.norm(b)
    c = O.cycle(A, b, None, None, None, S, tol, 10, 3, 2)
    assert c.converged and c.j == 3
    assert min(c.sres[:2]) > 1e-3 * np.linalg.norm(b)
    assert np.allclose(c.x_tilde, b / d, rtol=1e-9, atol=0)


def pin_harmonic_ritz_exact_with_a_sketch(O):
    pin_harmonic_ritz_exact_on_an_invariant_subspace(O, with_sketch=True)


PART_PINS = [pin_back_substitute_matches_library_triangular_solve, pin_sketched_ls_matches_library_least_squares,
             pin_numerical_rank_known_spectra_and_matrices, pin_select_largest_invariants,
             pin_select_largest_real_distinct_matches_sort, pin_invariant_basis_spans_an_invariant_subspace,
             pin_harmonic_ritz_exact_on_an_invariant_subspace, pin_harmonic_ritz_exact_with_a_sketch,
             pin_lucky_breakdown_stops_the_cycle, pin_finite_termination]


@pytest.mark.parametrize("pin", PART_PINS, ids=[f.__name__[4:] for f in PART_PINS])
def test_oracle_part(pin):
    pin(ORACLE)
