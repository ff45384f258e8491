"""Givens-sine residual estimator of sketched (augmented) GMRES.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the
product path.

Section 4.5 (Theorem on Givens sines and sketched GMRES angles): solving the
sketched least-squares problem by a progressive Givens QR of the sketched
Hessenberg matrix gives, at step j, a rotation whose sine is the sine of the
angle between S r_{j-1} and S A K_j, and the sketched residual norms obey
||S r_j|| = |s_j| ||S r_{j-1}||.  The Corollary that follows bounds the true
residual progressively through the unsketched sines and cosines:
||r_j|| <= sqrt((s_j^2 + 2 eps (1 + c_j)) / (1 - eps^2)) ||r_{j-1}||.

Section 5 extends this to the augmented cycle of Algorithm 1: with the
economy QR [S A U, S V_{j+1}] = W R (the basis whitening) and
G = R [[I, 0], [0, H]], the relation S A [U V_j] = W G holds with G upper
Hessenberg whose leading k x k block is already triangular, so the Givens QR
of G rotates only its Hessenberg part, one rotation per Arnoldi step.

The functions follow that construction in the paper's order: the QR of
[SAU, SV], the matrix G, then the rotations applied to the columns of G and
to the right-hand side W^T S r0 = beta R e_{k+1}.
"""
import numpy as np


def givens(a: float, b: float):
    """Rotation [[c, s], [-s, c]] with c a + s b = r >= 0 and -s a + c b = 0."""
    r = float(np.hypot(a, b))
    if r == 0.0:
        return 1.0, 0.0, 0.0
    return a / r, b / r, r


def sketched_g(SAU: np.ndarray, SV: np.ndarray, H: np.ndarray):
    """Section 5: R from the economy QR of [SAU, SV(:, 0:j+1)] and
    G = R blkdiag(I_k, H) (size (k + j + 1) x (k + j)); also returns R."""
    k = SAU.shape[1]
    j = H.shape[1]
    M = np.hstack([SAU, SV[:, :j + 1]])
    R = np.linalg.qr(M, mode="r")
    B = np.zeros((k + j + 1, k + j))
    B[:k, :k] = np.eye(k)
    B[k:, k:] = H[:j + 1, :j]
    return R @ B, R


def givens_sines(SAU: np.ndarray, SV: np.ndarray, H: np.ndarray, beta: float):
    """Progressive Givens QR of G (Section 5) with the right-hand side
    g = W^T S r0 = beta R(:, k) (S r0 = beta SV(:, 0), column k of [SAU, SV]).

    Returns per Arnoldi step j = 1..m the sine s_j and cosine c_j of the
    rotation that annihilates the subdiagonal entry of column k + j - 1, and
    the sketched residual norm ||S r_j|| read from the rotated right-hand side.
    The k columns of the triangular block need no rotation; rotating the
    Hessenberg part starts from the rhs rows k .. k + j."""
    k = SAU.shape[1]
    m = H.shape[1]
    G, R = sketched_g(SAU, SV, H)
    g = beta * R[:, k].copy()
    Gr = G.copy()
    sines, cosines, sres = [], [], []
    rots = []
    for j in range(m):
        col = k + j
        # previous rotations act on rows (k + i, k + i + 1) of this column
        for i, (c, s) in enumerate(rots):
            a, b = Gr[k + i, col], Gr[k + i + 1, col]
            Gr[k + i, col], Gr[k + i + 1, col] = c * a + s * b, -s * a + c * b
        c, s, r = givens(Gr[col, col], Gr[col + 1, col])
        Gr[col, col], Gr[col + 1, col] = r, 0.0
        a, b = g[col], g[col + 1]
        g[col], g[col + 1] = c * a + s * b, -s * a + c * b
        rots.append((c, s))
        sines.append(abs(s))
        cosines.append(abs(c))
        sres.append(abs(g[col + 1]))
    return np.array(sines), np.array(cosines), np.array(sres)


def corollary_factor(s: np.ndarray, c: np.ndarray, eps: float) -> np.ndarray:
    """Growth factor of the Corollary's progressive bound on the true residual:
    sqrt((s^2 + 2 eps (1 + c)) / (1 - eps^2))."""
    return np.sqrt((np.asarray(s) ** 2 + 2.0 * eps * (1.0 + np.asarray(c))) / (1.0 - eps * eps))
