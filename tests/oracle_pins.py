"""Checks that tie the GMRES-SDR oracle to results fixed outside itself.

Each pin takes the oracle module (``oracle.sdr`` or a copy with a planted
mistake) and raises AssertionError when the oracle disagrees with:
  * dense LU (numpy.linalg.solve) on small systems, including a sequence of
    perturbed systems with exact recycling (Section 3.6);
  * GMRES residual norms from an independent Householder-Arnoldi basis and
    numpy.linalg.lstsq when S = I (Section 2.1, eq. (sgmres) with S = I);
  * the augmented minimum-residual problem and the dense harmonic Ritz pencil
    when S = I (GMRES-DR special case, Sections 2.3 and 3.4);
  * the sketched Arnoldi relation solved with Givens rotations, the Givens-sine
    recurrence and the sGMRES/sFOM MR/OR identity (Section 4.5-4.6);
  * idempotency of the sketched residual projector (Lemma 4.1);
  * minimality of the sketched residual and the residual chain (eq. (reschain)).
"""
import numpy as np

import workloads as W
from oracle.sketch import Identity, SparseSign


def small_problem(n=12, conv=(10.0, 10.0)):
    A = W.make_cd2d(n, conv)
    return A, W.csr_to_dense(A), W.rhs(A.n)


def _orth(X):
    Q, _ = np.linalg.qr(X)
    return Q


def principal_angle_max(X, Y):
    Qx, Qy = _orth(X), _orth(Y)
    sv = np.linalg.svd(Qx.T @ Qy, compute_uv=False)
    return float(np.arccos(np.clip(sv.min(), -1.0, 1.0)))


def pin_dense_lu(sdr):
    A, D, b = small_problem(12)
    S = SparseSign(11, A.n, 60, 8)
    out = sdr.solve(A, b, S, m=20, k=5, t=2, rel_tol=1e-12, max_cycles=60)
    xs = np.linalg.solve(D, b)
    assert out.converged
    assert np.linalg.norm(out.x - xs) / np.linalg.norm(xs) < 1e-9
    assert np.linalg.norm(b - D @ out.x) <= 1e-12 * np.linalg.norm(b) * (1 + 1e-6)
    # 3D, 7-point
    A3 = W.make_cd3d(6, (20.0, 10.0, 5.0))
    D3 = W.csr_to_dense(A3)
    b3 = W.rhs(A3.n, 3)
    out3 = sdr.solve(A3, b3, SparseSign(12, A3.n, 80, 8), m=25, k=6, t=2, rel_tol=1e-12, max_cycles=60)
    xs3 = np.linalg.solve(D3, b3)
    assert out3.converged and np.linalg.norm(out3.x - xs3) / np.linalg.norm(xs3) < 1e-9


def pin_sequence_lu(sdr):
    A0, _, _ = small_problem(10)
    dvec = W.diag_perturbation(A0.n)
    As = list(W.sequence_matrices(A0, 4, 50.0, dvec))  # visible changes between systems
    bs = [W.rhs(A0.n, i) for i in range(4)]
    S = SparseSign(13, A0.n, 50, 8)
    outs = sdr.solve_sequence(As, bs, S, m=12, k=4, t=2, rel_tol=1e-11, max_cycles=80, record=True)
    Sd = S.dense()
    for i, (A, b, o) in enumerate(zip(As, bs, outs)):
        xs = np.linalg.solve(W.csr_to_dense(A), b)
        assert o.converged and np.linalg.norm(o.x - xs) / np.linalg.norm(xs) < 1e-8
        # every cycle starts from sketches consistent with the current A^(i):
        # SU = S U and SAU = S A^(i) U (the exact variant of Section 3.6)
        D = W.csr_to_dense(A)
        for c in o.cycle_log:
            U_in = c.info["U_in"]
            if U_in.shape[1]:
                ref = Sd @ D @ U_in
                assert np.allclose(c.info["SAU_in"], ref, rtol=0, atol=1e-9 * np.abs(ref).max()), i
                assert np.allclose(c.info["SU_in"], Sd @ U_in, rtol=0, atol=1e-9 * np.abs(c.info["SU_in"]).max())
    # the exact variant carries SU unchanged but SAU = S A^(i+1) U
    o = outs[-2]
    U, SU = o.U, o.SU
    assert np.allclose(S.apply_cols(U), SU, rtol=0, atol=1e-10 * np.abs(SU).max())


def _householder_krylov(D, r0, m):
    """Orthonormal bases of K_1..K_m from repeated library QR (independent of
    the oracle's truncated Gram-Schmidt)."""
    Q = (r0 / np.linalg.norm(r0))[:, None]
    bases = [Q]
    for _ in range(m - 1):
        Q, _ = np.linalg.qr(np.hstack([Q, D @ Q[:, -1:]]))
        bases.append(Q)
    return bases


def pin_gmres_identity_sketch(sdr):
    A, D, b = small_problem(12)
    m = 14
    for t in (2, m):
        c = sdr.cycle(A, b, None, None, None, Identity(A.n), 0.0, m, t, 3, record=True)
        bases = _householder_krylov(D, b, m)
        for j in range(m):
            K = bases[j]
            y, *_ = np.linalg.lstsq(D @ K, b, rcond=None)
            ref = np.linalg.norm(b - D @ K @ y)
            assert abs(c.sres[j] - ref) <= 1e-9 * ref + 1e-12 * np.linalg.norm(b), (t, j, c.sres[j], ref)


def _dense_harmonic(D, Wb, k):
    """Harmonic Ritz pairs of A over span(Wb): (A Wb)^+ Wb y = mu y, k largest |mu|."""
    M, *_ = np.linalg.lstsq(D @ Wb, Wb, rcond=None)
    mu, Y = np.linalg.eig(M)
    order = np.argsort(-np.abs(mu), kind="stable")
    return mu, Y, order


def pin_gmres_dr_identity_sketch(sdr):
    A, D, b = small_problem(12, (30.0, 10.0))
    m, k = 12, 4
    out = sdr.solve(A, b, Identity(A.n), m=m, k=k, t=2, rel_tol=1e-13, max_cycles=5, record=True)
    assert len(out.cycle_log) >= 3
    for ci, c in enumerate(out.cycle_log):
        inf = c.info
        r0 = inf["Sr0"]  # S = I
        U0 = inf["U_in"]
        if ci > 0:
            assert U0.shape[1] >= k
            # SAU carried over must be A U exactly (S = I)
            assert np.allclose(inf["SAU_in"], D @ U0, rtol=0, atol=1e-10 * np.abs(D @ U0).max())
        for j in range(c.j):
            Wj = np.hstack([U0, inf["V"][:, :j + 1]])
            y, *_ = np.linalg.lstsq(D @ Wj, r0, rcond=None)
            ref = np.linalg.norm(r0 - D @ Wj @ y)
            assert abs(c.sres[j] - ref) <= 1e-8 * ref + 1e-12 * np.linalg.norm(r0), (ci, j)
        # harmonic Ritz values and vectors of the dense pencil
        Wb = np.hstack([U0, inf["V"][:, :c.j]])
        mu, Y, order = _dense_harmonic(D, Wb, k)
        hr = inf["hr"]
        kk = len(hr["sel"])
        got = np.sort(np.abs(hr["mu"][hr["sel"]]))[::-1]
        ref = np.abs(mu[order[:kk]])
        assert np.allclose(got, ref, rtol=1e-8), (got, ref)
        # span of the new U = span of the selected harmonic Ritz vectors
        sel = order[:kk]
        vecs = []
        for i in sel:
            if mu[i].imag == 0:
                vecs.append(Y[:, i].real)
            elif mu[i].imag > 0:  # one member of each conjugate pair gives Re and Im
                vecs += [Y[:, i].real, Y[:, i].imag]
        ref_span = Wb @ np.stack(vecs, axis=1)
        assert ref_span.shape[1] == c.U.shape[1]
        assert principal_angle_max(c.U, ref_span) < 1e-7


def pin_augmented_without_sketches(sdr):
    """Algorithm 1 with U given but SU, SAU not provided: they are computed
    first, and with S = I every sres is the augmented minimum residual."""
    A, D, b = small_problem(12)
    U = np.random.default_rng(5).standard_normal((A.n, 3))
    c = sdr.cycle(A, b, U, None, None, Identity(A.n), 0.0, 10, 2, 3, record=True)
    for j in range(c.j):
        Wj = np.hstack([U, c.info["V"][:, :j + 1]])
        y, *_ = np.linalg.lstsq(D @ Wj, b, rcond=None)
        ref = np.linalg.norm(b - D @ Wj @ y)
        assert abs(c.sres[j] - ref) <= 1e-8 * ref + 1e-12 * np.linalg.norm(b), j


def _givens_ls(Hh, g):
    """Progressive Givens QR of the (j+1) x j upper-Hessenberg Hh (textbook GMRES)."""
    mm = Hh.shape[1]
    R = Hh.copy()
    gg = g.copy()
    cs, sn, res = [], [], []
    for j in range(mm):
        for i in range(j):
            a, bb = R[i, j], R[i + 1, j]
            R[i, j] = cs[i] * a + sn[i] * bb
            R[i + 1, j] = -sn[i] * a + cs[i] * bb
        a, bb = R[j, j], R[j + 1, j]
        rho = np.hypot(a, bb)
        c_, s_ = a / rho, bb / rho
        cs.append(c_)
        sn.append(s_)
        R[j, j], R[j + 1, j] = rho, 0.0
        gg[j], gg[j + 1] = c_ * gg[j], -s_ * gg[j]
        res.append(abs(gg[j + 1]))
    return R, gg, np.array(cs), np.array(sn), np.array(res)


def pin_sketched_arnoldi_mr_or(sdr):
    A = W.make_cd2d(24, (10.0, 10.0))
    b = W.rhs(A.n)
    S = SparseSign(21, A.n, 120, 8)
    m = 30
    c = sdr.cycle(A, b, None, None, None, S, 0.0, m, 2, 5, record=True)
    V, H, SV = c.info["V"], c.info["H"], c.info["SV"]
    # sketched Arnoldi relation SAV = W_hat H_hat (Section 4.5)
    Wh, Rsv = np.linalg.qr(SV)
    Hh = Rsv @ H
    g = Wh.T @ c.info["Sr0"]
    _, gg, cs, sn, res = _givens_ls(Hh, g)
    sres = np.array(c.sres)
    nS = np.linalg.norm(c.info["Sr0"])
    assert np.all(np.abs(sres - res) <= 1e-8 * res + 1e-12 * nS), np.max(np.abs(sres - res) / res)
    # Givens sine recurrence ||S r_j|| = |s_j| ||S r_{j-1}||
    prev = np.concatenate([[nS], res[:-1]])
    assert np.allclose(res, np.abs(sn) * prev, rtol=1e-10)
    # sGMRES / sFOM MR/OR identity x_G(j) = c_j^2 x_F(j) + s_j^2 x_G(j-1)
    def yG(j):
        y, *_ = np.linalg.lstsq(Hh[:j + 1, :j], g[:j + 1], rcond=None)
        return V[:, :j] @ y
    for j in range(2, m + 1, 4):
        yF = np.linalg.solve(Hh[:j, :j], g[:j])
        xF = V[:, :j] @ yF
        lhs = yG(j)
        rhs = cs[j - 1] ** 2 * xF + sn[j - 1] ** 2 * yG(j - 1)
        assert np.linalg.norm(lhs - rhs) <= 1e-8 * np.linalg.norm(lhs)
    # the oracle's final correction is the sGMRES iterate
    assert np.linalg.norm(c.x_tilde - yG(m)) <= 1e-8 * np.linalg.norm(c.x_tilde)


def pin_projector_and_minimality(sdr):
    A, D, b = small_problem(10)
    S = SparseSign(31, A.n, 40, 8)
    Sd = S.dense()
    c = sdr.cycle(A, b, None, None, None, S, 0.0, 12, 2, 3, record=True)
    V, SAV, Sr0 = c.info["V"][:, :c.j], c.info["SAV"], c.info["Sr0"]
    # the sketched image is S A V (eq. (truncated-sketched-Arnoldi))
    assert np.allclose(SAV, Sd @ D @ V, rtol=0, atol=1e-9 * np.abs(SAV).max())
    Phi = D @ V @ np.linalg.pinv(SAV) @ Sd
    assert np.linalg.norm(Phi @ Phi - Phi) <= 1e-7 * np.linalg.norm(Phi)  # Lemma 4.1
    y = c.info["y"]
    rs = Sr0 - SAV @ y
    assert np.linalg.norm(SAV.T @ rs) <= 1e-9 * np.linalg.norm(SAV) * np.linalg.norm(Sr0)
    assert abs(np.linalg.norm(rs) - c.sres[-1]) <= 1e-12 * np.linalg.norm(Sr0)
    rng = np.random.default_rng(2)
    for _ in range(200):
        yp = y + 1e-3 * np.linalg.norm(y) * rng.standard_normal(y.size) / np.sqrt(y.size)
        assert np.linalg.norm(Sr0 - SAV @ yp) >= c.sres[-1] * (1 - 1e-12)


def pin_residual_chain(sdr):
    A, D, b = small_problem(20)
    S = SparseSign(41, A.n, 240, 8)
    Sd = S.dense()
    c = sdr.cycle(A, b, None, None, None, S, 0.0, 10, 2, 3, record=True)
    V = c.info["V"][:, :c.j]
    AV = D @ V
    r_t = b - AV @ c.info["y"]  # sketched-GMRES residual
    yg, *_ = np.linalg.lstsq(AV, b, rcond=None)
    r_g = b - AV @ yg  # full-GMRES residual over the same space
    Q = _orth(np.hstack([b[:, None], AV]))
    sv = np.linalg.svd(Sd @ Q, compute_uv=False)
    eps = max(1 - sv.min() ** 2, sv.max() ** 2 - 1)
    assert eps < 1
    lo, hi = np.sqrt(1 - eps), np.sqrt(1 + eps)
    n_g, n_t = np.linalg.norm(r_g), np.linalg.norm(r_t)
    tiny = 1e-12 * np.linalg.norm(b)
    assert n_g <= n_t + tiny
    assert n_t <= np.linalg.norm(Sd @ r_t) / lo + tiny
    assert np.linalg.norm(Sd @ r_t) <= np.linalg.norm(Sd @ r_g) + tiny
    assert np.linalg.norm(Sd @ r_g) / lo <= hi / lo * n_g + tiny
    assert abs(np.linalg.norm(Sd @ r_t) - c.sres[-1]) <= 1e-10 * np.linalg.norm(b)


ALL_PINS = [pin_dense_lu, pin_sequence_lu, pin_gmres_identity_sketch, pin_gmres_dr_identity_sketch,
            pin_augmented_without_sketches,
            pin_sketched_arnoldi_mr_or, pin_projector_and_minimality, pin_residual_chain]
