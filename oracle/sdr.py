"""GMRES-SDR in plain FP64, step by step as the paper states it.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the
product path.

Algorithm 1 (one cycle), Section 3.4 (residual control with `safety`),
Section 3.5 (sketched harmonic Ritz extraction with a truncated SVD and an
ordered QZ), Section 3.6 (sequences: fixed A with varying b, and the exact and
inexact variants for varying A).

Readings where the paper is silent or garbled (each one is listed in the
design notes of the repository):
  * the zero blocks of SV in Algorithm 1 are s x m (printed as N x m);
  * "SW" in the M_ell line is S[U, V] = [SU, SV(:, 1:j)] (Section 3.5);
  * after an early break the recycle update uses the j columns actually built;
  * ell = #{sigma_i > sigma_1 * d * eps}, d the number of columns of SAW;
  * QZ of (M_ell, Sigma_ell) is taken through the eigenpairs of
    Sigma_ell^{-1} M_ell: the span of Z(:, 1:k) is the span of the real and
    imaginary parts of the selected eigenvectors;
  * k largest |mu| are kept (ties: larger real part, then lower index); a
    complex-conjugate pair is kept whole, so a pair at the k-th place gives
    k+1 columns;
  * `safety` starts from its default at every cycle;
  * an exactly zero H(j+1, j) forces the true-residual check at that j;
  * tol is absolute: tol = rel_tol * ||b||.

Parity unpinned: the selection when |mu_k| and |mu_{k+1}| nearly tie, and the
basis of U (only its span is determined); see the package docstring.
"""
from dataclasses import dataclass, field

import numpy as np

EPS = np.finfo(np.float64).eps


def csr_matvec(A, x: np.ndarray) -> np.ndarray:
    """y = A x for a CSR matrix (rowptr, col, val)."""
    rows = _row_index(A)
    return np.bincount(rows, weights=A.val * x[A.col], minlength=A.n)


def _row_index(A):
    cache = getattr(A, "_oracle_rows", None)
    if cache is None or cache.shape[0] != A.val.shape[0]:
        cache = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.rowptr.astype(np.int64)))
        try:
            A._oracle_rows = cache
        except AttributeError:
            pass
    return cache


def csr_matmat(A, X: np.ndarray) -> np.ndarray:
    return np.stack([csr_matvec(A, X[:, i]) for i in range(X.shape[1])], axis=1) \
        if X.shape[1] else np.zeros((A.n, 0))


def back_substitute(R: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Solve R y = z for upper-triangular R (the R^{-1} of Algorithm 1)."""
    n = R.shape[0]
    y = np.zeros(n)
    for i in range(n - 1, -1, -1):
        y[i] = (z[i] - R[i, i + 1:] @ y[i + 1:]) / R[i, i]
    return y


def sketched_ls(SAW: np.ndarray, Sr0: np.ndarray):
    """Algorithm 1, QR-based least squares: [Q, R] = qr(SAW) (Householder,
    economic), y = R^{-1} Q^* S r0, sres = ||S r0 - SAW y|| taken directly
    from the residual vector."""
    Q, R = np.linalg.qr(SAW, mode="reduced")
    y = back_substitute(R, Q.T @ Sr0)
    sres = float(np.linalg.norm(Sr0 - SAW @ y))
    return y, sres


def sau_rank_deficient(SAU: np.ndarray) -> bool:
    """Whether a sketched recycle block SAU (s x kd) is numerically
    rank-deficient for Algorithm 1's least squares, which needs R^{-1} from the
    QR of SAW = [SAU, SAV].  Reading (the paper is silent): deficient when some
    diagonal entry of R in SAU = QR has |R_pp| <= s * eps * max_q ||SAU(:, q)||,
    or a value is not finite."""
    if SAU.shape[1] == 0:
        return False
    if not np.all(np.isfinite(SAU)):
        return True
    s = SAU.shape[0]
    maxn = float(np.max(np.linalg.norm(SAU, axis=0)))
    if maxn == 0.0:
        return True
    R = np.linalg.qr(SAU, mode="r")
    return bool(np.any(np.abs(np.diag(R)) <= s * EPS * maxn))


def numerical_rank(sig: np.ndarray, d: int) -> int:
    """ell = #{sigma_i > sigma_1 * d * eps} (truncated economic SVD, Section 3.5)."""
    if sig.size == 0 or sig[0] == 0.0:
        return 0
    return int(np.count_nonzero(sig > sig[0] * d * EPS))


def select_largest(mu: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k eigenvalues of largest modulus (ties: larger real part,
    then lower index; Section 3.5 targets the largest-modulus mu).  A complex
    eigenvalue is taken together with a conjugate partner, so a pair at the
    k-th place gives k + 1 indices (the real basis of Section 3.5 needs whole
    pairs; this also holds when a pair is repeated exactly)."""
    idx = np.arange(mu.size)
    order = np.lexsort((idx, -mu.real, -np.abs(mu)))
    kk = min(k, mu.size)
    sel, used = [], np.zeros(mu.size, dtype=bool)
    for i in order:
        if len(sel) >= kk:
            break
        if used[i]:
            continue
        sel.append(i)
        used[i] = True
        if mu[i].imag != 0.0:
            for j in order:  # the partner: same modulus and real part, later in the order
                if not used[j] and mu[j] == np.conj(mu[i]):
                    sel.append(j)
                    used[j] = True
                    break
    return np.array(sel, dtype=np.int64)


def invariant_basis(mu: np.ndarray, Y: np.ndarray, sel: np.ndarray) -> np.ndarray:
    """Orthonormal real basis of the span of the selected eigenvectors
    (a conjugate pair contributes the real and imaginary part of one member)."""
    cols, used = [], set()
    for i in sel:
        i = int(i)
        if i in used:
            continue
        if mu[i].imag == 0.0:
            cols.append(Y[:, i].real)
            used.add(i)
        else:
            partner = [j for j in sel if int(j) != i and int(j) not in used and mu[j] == np.conj(mu[i])]
            cols.append(Y[:, i].real)
            cols.append(Y[:, i].imag)
            used.add(i)
            if partner:
                used.add(int(partner[0]))
    if not cols:
        return np.zeros((Y.shape[0], 0))
    Z, _ = np.linalg.qr(np.stack(cols, axis=1), mode="reduced")
    return Z


def harmonic_ritz_update(SAW, SW, k):
    """Section 3.5 / Algorithm 1 recycling block.

    Truncated SVD SAW ~ U_l Sigma_l V_l^*, M_l = U_l^* (S[U V]) V_l, ordered QZ
    of (M_l, Sigma_l) with the k largest-modulus eigenvalues first; returns
    P = V_l Z(:, 1:k) together with the intermediate quantities."""
    d = SAW.shape[1]
    Uh, sig, Vt = np.linalg.svd(SAW, full_matrices=False)
    ell = numerical_rank(sig, d)
    Ul, sl, Vl = Uh[:, :ell], sig[:ell], Vt[:ell, :].T
    M = Ul.T @ SW @ Vl
    B = M / sl[:, None]  # Sigma_l^{-1} M_l: its eigenpairs are those of the pencil (M_l, Sigma_l)
    mu, Yv = np.linalg.eig(B)
    sel = select_largest(mu, k)
    Z = invariant_basis(mu, Yv, sel)
    P = Vl @ Z
    return P, dict(sig=sig, ell=ell, M=M, mu=mu, sel=sel, Z=Z, Vl=Vl, Ul=Ul)


@dataclass
class Cycle:
    x_tilde: np.ndarray
    r: np.ndarray  # r0 - A x_tilde (the vector whose norm is the last res)
    res: float
    converged: bool
    j: int  # Krylov columns built (j_f)
    sres: list  # sketched residual after each Arnoldi step
    checks: list  # (j, sres, res) at each true-residual evaluation
    safety: float
    U: np.ndarray
    SU: np.ndarray
    SAU: np.ndarray
    matvecs: int
    info: dict = field(default_factory=dict)


def cycle(A, r0, U, SU, SAU, S, tol, m, t, k, safety=1.4, record=False) -> Cycle:
    """One cycle of Algorithm 1 for A x = r0 (the correction equation).

    Krylov columns are 0-based here: V[:, 0] = r0/||r0||, step j (0..m-1)
    builds V[:, j+1] and SAW gains its (k_hat + j)-th column."""
    N = A.n
    s = S.s
    matvecs = 0
    if U is None or U.shape[1] == 0:
        U = np.zeros((N, 0))
        SU = np.zeros((s, 0))
        SAU = np.zeros((s, 0))
    else:
        if SU is None:  # line "compute sketches SU and SAU if not provided"
            SU = S.apply_cols(U)
        if SAU is None:
            SAU = S.apply_cols(csr_matmat(A, U))
            matvecs += U.shape[1]
    kh = U.shape[1]
    Sr0 = S.apply(r0)  # sketch the initial residual
    beta = float(np.linalg.norm(r0))
    V = np.zeros((N, m + 1))
    V[:, 0] = r0 / beta
    H = np.zeros((m + 1, m))
    SV = np.zeros((s, m + 1))
    SV[:, 0] = Sr0 / beta
    SAV = np.zeros((s, m))
    sres_hist, checks = [], []
    x_tilde = None
    r = None
    res = np.inf
    converged = False
    jf = m
    y = None
    for j in range(m):
        w = csr_matvec(A, V[:, j])  # w := A V(:, j)
        matvecs += 1
        for i in range(max(j - t + 1, 0), j + 1):  # truncated MGS over the last t vectors
            H[i, j] = V[:, i] @ w
            w = w - V[:, i] * H[i, j]
        H[j + 1, j] = np.linalg.norm(w)
        breakdown = H[j + 1, j] == 0.0
        V[:, j + 1] = 0.0 if breakdown else w / H[j + 1, j]
        SV[:, j + 1] = S.apply(V[:, j + 1])  # one sketch per iteration
        SAV[:, j] = SV[:, :j + 2] @ H[:j + 2, j]  # sketched image, no extra sketch
        SAW = np.hstack([SAU, SAV[:, :j + 1]])
        y, sres = sketched_ls(SAW, Sr0)
        sres_hist.append(sres)
        if sres < tol / safety or j == m - 1 or breakdown:
            x_tilde = np.hstack([U, V[:, :j + 1]]) @ y
            r = r0 - csr_matvec(A, x_tilde)  # true residual
            matvecs += 1
            res = float(np.linalg.norm(r))
            checks.append((j, sres, res))
            if res < tol:
                converged = True
                jf = j + 1
                break
            safety = res / sres  # increase the safety factor
            if breakdown:
                jf = j + 1
                break
    # Recycling block (Section 3.5) over the columns actually built.
    SAW = np.hstack([SAU, SAV[:, :jf]])
    SW = np.hstack([SU, SV[:, :jf]])
    P, hr = harmonic_ritz_update(SAW, SW, k)
    U_new = np.hstack([U, V[:, :jf]]) @ P
    SU_new = SW @ P
    SAU_new = SAW @ P
    info = dict(hr=hr, y=y)
    if record:
        info.update(V=V[:, :jf + 1], H=H[:jf + 1, :jf], SV=SV[:, :jf + 1], SAV=SAV[:, :jf],
                    Sr0=Sr0, beta=beta, SAW=SAW, SW=SW, P=P, U_in=U, SU_in=SU, SAU_in=SAU)
    return Cycle(x_tilde, r, res, converged, jf, sres_hist, checks, safety,
                 U_new, SU_new, SAU_new, matvecs, info)


@dataclass
class Solve:
    x: np.ndarray
    converged: bool
    cycles: int
    res: float
    tol: float
    sres_per_cycle: list  # list of per-step sres lists
    checks: list
    U: np.ndarray
    SU: np.ndarray
    SAU: np.ndarray
    matvecs: int
    cycle_log: list = field(default_factory=list)
    sau_refreshes: int = 0


STALE_RATIO = 4.0  # res > STALE_RATIO * sres at a cycle's last check marks SAU stale


def solve(A, b, S, m, k, t, rel_tol, safety0=1.4, max_cycles=200, U=None, SU=None, SAU=None,
          x0=None, persist_safety=False, record=False, cycle_hook=None, stale_check=False) -> Solve:
    """Restarted GMRES-SDR for A x = b: repeat Algorithm 1 on the current
    residual, x <- x + x_tilde, r0 <- r0 - A x_tilde, until res < tol.

    stale_check (failure detection for the inexact variant of Section 3.6):
    with an exact SAU = S A U the true residual r lies in the subspace the
    sketch embeds, so ||r|| <= ||S r|| / (1 - eps) (Section 3, Eq. (sketch)),
    i.e. res <= 4 sres for any eps <= 3/4.  When a cycle ends unconverged with
    res > 4 sres at its last check, SAU can only be stale: SAU of the new
    recycle space is then recomputed as S A U (k products) before the next
    cycle."""
    N = A.n
    x = np.zeros(N) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    tol = rel_tol * float(np.linalg.norm(b))
    r = b - csr_matvec(A, x) if x0 is not None else np.array(b, dtype=np.float64, copy=True)
    matvecs = 1 if x0 is not None else 0
    res = float(np.linalg.norm(r))
    sres_all, checks_all, log = [], [], []
    safety = safety0
    cycles = 0
    refreshes = 0
    converged = res < tol
    while not converged and cycles < max_cycles:
        if cycle_hook is not None:
            cycle_hook(cycles, x, r, U, SU, SAU, safety)
        c = cycle(A, r, U, SU, SAU, S, tol, m, t, k, safety=safety, record=record)
        cycles += 1
        matvecs += c.matvecs
        x = x + c.x_tilde
        r = c.r
        res = c.res
        U, SU, SAU = c.U, c.SU, c.SAU
        sres_all.append(c.sres)
        checks_all.append(c.checks)
        if record:
            log.append(c)
        safety = c.safety if persist_safety else safety0
        converged = c.converged
        if (stale_check and not converged and cycles < max_cycles and U.shape[1] and c.checks
                and c.checks[-1][2] > STALE_RATIO * c.checks[-1][1]):
            SAU = S.apply_cols(csr_matmat(A, U))
            matvecs += U.shape[1]
            refreshes += 1
    return Solve(x, converged, cycles, res, tol, sres_all, checks_all, U, SU, SAU, matvecs, log, refreshes)


def solve_sequence(As, bs, S, m, k, t, rel_tol, exact=True, fixed_matrix=False, **kw):
    """Section 3.6: carry U, SU, SAU from system i to i+1.

    fixed_matrix: A is the same for every system, so U, SU, SAU are reused as
    they are.  Otherwise the exact variant recomputes SAU = S A^(i+1) U with k
    matrix-vector products and sketches; the inexact one keeps S A^(i) U."""
    U = SU = SAU = None
    out = []
    for i, (A, b) in enumerate(zip(As, bs)):
        if i > 0 and U is not None and U.shape[1] and exact and not fixed_matrix:
            SAU = S.apply_cols(csr_matmat(A, U))
        res = solve(A, b, S, m, k, t, rel_tol, U=U, SU=SU, SAU=SAU, **kw)
        if i > 0 and U is not None and U.shape[1] and exact and not fixed_matrix:
            res.matvecs += U.shape[1]
        U, SU, SAU = res.U, res.SU, res.SAU
        out.append(res)
    return out
