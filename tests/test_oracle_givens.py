"""Pins of the oracle's Givens-sine residual estimator (Section 4.5, Theorem
on Givens sines and its Corollary; Section 5, the augmented cycle).

Fixed outside the estimator:
  * its sketched residual norms equal those of the cycle's Householder least
    squares (a different factorisation of a different matrix, SAW);
  * with S = I, t = m and no recycling its sines are textbook GMRES's: the
    ratios of consecutive GMRES residual norms, from independent Householder
    Krylov bases and numpy.linalg.lstsq;
  * each sine is the sine of the angle between S r_{j-1} and S A [U V_j],
    computed from principal angles;
  * the Corollary's progressive bound holds for the true residuals, with
    eps the measured distortion of S on span[r0, A U, A V]."""
import numpy as np
import pytest

import workloads as W
from oracle import givens as G
from oracle import sdr as O
from oracle.sketch import Identity, SparseSign


def _cycles(n=12, s=60, m=16, k=4, t=2):
    """A first cycle and a recycled second cycle of a 2D problem, recorded."""
    A = W.make_cd2d(n, (10.0, 10.0))
    b = W.rhs(A.n)
    S = SparseSign(17, A.n, s, 8)
    c1 = O.cycle(A, b, None, None, None, S, 0.0, m, t, k, record=True)
    r1 = b - O.csr_matvec(A, c1.x_tilde)
    c2 = O.cycle(A, r1, c1.U, c1.SU, c1.SAU, S, 0.0, m, t, k, record=True)
    return A, S, (b, c1), (r1, c2)


def test_estimator_sres_equals_householder_least_squares():
    A, S, first, second = _cycles()
    for r0, c in (first, second):
        info = c.info
        s, co, sres = G.givens_sines(info["SAU_in"], info["SV"], info["H"], info["beta"])
        ref = np.asarray(c.sres)
        assert np.allclose(sres, ref, rtol=1e-10, atol=1e-13 * np.linalg.norm(info["Sr0"]))
        assert np.allclose(s ** 2 + co ** 2, 1.0, atol=1e-14)
        # the Theorem's recurrence ||S r_j|| = |s_j| ||S r_{j-1}||
        prev = np.concatenate([[np.linalg.norm(info["Sr0"] - info["SAU_in"] @ np.linalg.lstsq(
            info["SAU_in"], info["Sr0"], rcond=None)[0]) if info["SAU_in"].shape[1] else np.linalg.norm(
            info["Sr0"])], ref[:-1]])
        assert np.allclose(ref, s * prev, rtol=1e-9)


def _householder_krylov(D, r0, m):
    Q = (r0 / np.linalg.norm(r0))[:, None]
    bases = [Q]
    for _ in range(m - 1):
        Q, _ = np.linalg.qr(np.hstack([Q, D @ Q[:, -1:]]))
        bases.append(Q)
    return bases


def test_identity_sketch_gives_textbook_gmres_sines():
    A = W.make_cd2d(12, (10.0, 10.0))
    D = W.csr_to_dense(A)
    b = W.rhs(A.n)
    m = 14
    c = O.cycle(A, b, None, None, None, Identity(A.n), 0.0, m, m, 3, record=True)
    s, co, sres = G.givens_sines(c.info["SAU_in"], c.info["SV"], c.info["H"], c.info["beta"])
    res = [np.linalg.norm(b)]
    for K in _householder_krylov(D, b, m):
        y, *_ = np.linalg.lstsq(D @ K, b, rcond=None)
        res.append(np.linalg.norm(b - D @ K @ y))
    res = np.asarray(res)
    assert np.allclose(s, res[1:] / res[:-1], rtol=1e-9)
    assert np.allclose(sres, res[1:], rtol=1e-9)


def _sin_angle(v, M):
    """Sine of the angle between vector v and range(M)."""
    Q, _ = np.linalg.qr(M)
    p = Q @ (Q.T @ v)
    return np.linalg.norm(v - p) / np.linalg.norm(v)


def test_sines_are_sketched_subspace_angles():
    A, S, first, (r0, c) = _cycles()
    info = c.info
    s, co, _ = G.givens_sines(info["SAU_in"], info["SV"], info["H"], info["beta"])
    SAU, SAV, Sr0 = info["SAU_in"], info["SAV"], info["Sr0"]
    Sr_prev = Sr0 - SAU @ np.linalg.lstsq(SAU, Sr0, rcond=None)[0]
    for j in range(SAV.shape[1]):
        SAW = np.hstack([SAU, SAV[:, :j + 1]])
        assert abs(s[j] - _sin_angle(Sr_prev, SAW)) <= 1e-9, j
        y = np.linalg.lstsq(SAW, Sr0, rcond=None)[0]
        Sr_prev = Sr0 - SAW @ y


def test_corollary_bound_on_true_residuals():
    """||r_j|| <= factor(s_j, c_j, eps) ||r_{j-1}|| with the unsketched sines
    and cosines of the angles between r_{j-1} and A [U V_j], and eps the
    distortion of S on span[r0, A U, A V] (Section 3, Eq. (sketch)); a sketch
    of 16 times the subspace dimension keeps eps below one."""
    A, S, first, (r0, c) = _cycles(n=24, s=360, m=16, k=4)
    info = c.info
    U, V = info["U_in"], info["V"]
    m = info["SAV"].shape[1]
    AW = O.csr_matmat(A, np.hstack([U, V[:, :m]]))
    Q, _ = np.linalg.qr(np.hstack([r0[:, None], AW]))
    sv = np.linalg.svd(S.apply_cols(Q), compute_uv=False)
    eps = max(abs(sv.max() ** 2 - 1.0), abs(1.0 - sv.min() ** 2))
    assert eps < 1.0
    SAU, SAV, Sr0 = info["SAU_in"], info["SAV"], info["Sr0"]
    k = U.shape[1]
    r_prev = r0 - AW[:, :k] @ np.linalg.lstsq(SAU, Sr0, rcond=None)[0]
    for j in range(m):
        SAW = np.hstack([SAU, SAV[:, :j + 1]])
        y = np.linalg.lstsq(SAW, Sr0, rcond=None)[0]
        r = r0 - AW[:, :k + j + 1] @ y
        sj = _sin_angle(r_prev, AW[:, :k + j + 1])
        cj = np.sqrt(max(0.0, 1.0 - sj * sj))
        bound = G.corollary_factor(sj, cj, eps) * np.linalg.norm(r_prev)
        assert np.linalg.norm(r) <= bound * (1 + 1e-12), (j, np.linalg.norm(r), bound)
        r_prev = r


@pytest.mark.parametrize("flip", ["sign", "offset"])
def test_planted_mistakes_are_caught(flip, monkeypatch):
    """A wrong rotation sign, or the triangular block taken one column short
    (the rotations then start one row off), break the equality with the
    Householder least squares."""
    A, S, first, (r0, c) = _cycles()
    info = c.info
    orig = G.givens

    if flip == "sign":
        def bad(a, b):
            cc, ss, r = orig(a, b)
            return cc, -ss, r
        monkeypatch.setattr(G, "givens", bad)
        s, co, sres = G.givens_sines(info["SAU_in"], info["SV"], info["H"], info["beta"])
    else:
        SAU = info["SAU_in"]
        s, co, sres = G.givens_sines(SAU[:, :-1], info["SV"], info["H"], info["beta"])
    assert not np.allclose(sres, np.asarray(c.sres), rtol=1e-6)
