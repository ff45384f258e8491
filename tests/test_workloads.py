"""The seeded synthetic inputs against their definitions (CPU only).

Each stencil is compared on a small grid with a dense matrix assembled
independently from Kronecker products of 1-D difference matrices; the paper's
own operator (Section 6.3) against its printed formula; the variable-coefficient
operator against its constant-coefficient special case and the symmetry of its
diffusion part; the nonzero counts of the benchmark sizes against their closed
forms; and the random inputs for determinism and their stated distributions."""
import numpy as np
import pytest

import workloads as W


def tridiag(n, sub, diag, sup):
    return np.diag(np.full(n, float(diag))) + np.diag(np.full(n - 1, float(sub)), -1) + \
        np.diag(np.full(n - 1, float(sup)), 1)


def upwind_1d(n, c, h):
    """c d/dx by first-order upwind: backward difference for c > 0, forward for c < 0."""
    if c >= 0:
        return c / h * tridiag(n, -1, 1, 0)
    return c / h * tridiag(n, 0, -1, 1)


def check_csr_structure(A):
    rp = A.rowptr.astype(np.int64)
    assert rp[0] == 0 and np.all(np.diff(rp) >= 1) and rp[-1] == A.col.size == A.val.size
    rows = np.repeat(np.arange(A.n), np.diff(rp))
    assert np.count_nonzero(A.col == rows) == A.n  # every row stores its diagonal
    for r in range(A.n):  # columns strictly ascending within a row
        assert np.all(np.diff(A.col[rp[r]:rp[r + 1]]) > 0)


@pytest.mark.parametrize("conv", [(10.0, 10.0), (3.0, -7.0), (0.0, 25.0)])
def test_cd2d_equals_kronecker_definition(conv):
    n, diff = 5, 1.0
    h = 1.0 / (n + 1)
    I = np.eye(n)
    T = diff / h**2 * tridiag(n, -1, 2, -1)
    ref = np.kron(I, T) + np.kron(T, I) + np.kron(I, upwind_1d(n, conv[0], h)) + \
        np.kron(upwind_1d(n, conv[1], h), I)  # x fastest: x acts within a row of the grid
    A = W.make_cd2d(n, conv)
    check_csr_structure(A)
    assert np.allclose(W.csr_to_dense(A), ref, rtol=1e-14, atol=1e-9)


@pytest.mark.parametrize("conv", [(20.0, 10.0, 5.0), (-4.0, 9.0, -2.0)])
def test_cd3d_equals_kronecker_definition(conv):
    n = 4
    h = 1.0 / (n + 1)
    I = np.eye(n)
    T = tridiag(n, -1, 2, -1) / h**2
    ref = np.kron(I, np.kron(I, T)) + np.kron(I, np.kron(T, I)) + np.kron(T, np.kron(I, I)) + \
        np.kron(I, np.kron(I, upwind_1d(n, conv[0], h))) + np.kron(I, np.kron(upwind_1d(n, conv[1], h), I)) + \
        np.kron(upwind_1d(n, conv[2], h), np.kron(I, I))
    A = W.make_cd3d(n, conv)
    check_csr_structure(A)
    assert np.allclose(W.csr_to_dense(A), ref, rtol=1e-14, atol=1e-9)


def test_benchmark_sizes_nonzero_counts():
    """5n^2 - 4n entries in 2D and 7n^3 - 6n^2 in 3D (the boundary drops one
    neighbour per face); the 64^2 and 128^3 workloads."""
    A = W.make_cd2d(64)
    assert (A.n, A.nnz) == (4096, 5 * 64**2 - 4 * 64) == (4096, 20224)
    A = W.make_cd3d(128)
    assert (A.n, A.nnz) == (2097152, 7 * 128**3 - 6 * 128**2) == (2097152, 14581760)
    assert A.rowptr.dtype == np.int32 and A.col.dtype == np.int32 and A.val.dtype == np.float64


@pytest.mark.parametrize("alpha", [0.0, 5.0, 20.0])
def test_paper_operator_section_6_3(alpha):
    """(L (x) I + I (x) L) + alpha (D (x) I + I (x) D), L = (n+1)^2 tridiag(1, -2, 1),
    D = (n+1)/2 tridiag(-1, 0, 1)."""
    n = 6
    I = np.eye(n)
    L = (n + 1) ** 2 * tridiag(n, 1, -2, 1)
    D = (n + 1) / 2.0 * tridiag(n, -1, 0, 1)
    ref = np.kron(L, I) + np.kron(I, L) + alpha * (np.kron(D, I) + np.kron(I, D))
    A = W.make_cd_paper(n, alpha)
    check_csr_structure(A)
    assert np.allclose(W.csr_to_dense(A), ref, rtol=1e-14, atol=1e-9)


def test_vcdiff_constant_field_is_the_upwind_stencil():
    n = 7
    A = W.make_vcdiff(n, np.zeros(n * n), (10.0, -3.0))
    assert np.allclose(W.csr_to_dense(A), W.csr_to_dense(W.make_cd2d(n, (10.0, -3.0))), rtol=1e-14, atol=1e-9)


def test_vcdiff_diffusion_part_is_symmetric_and_conservative():
    n = 8
    theta = np.random.default_rng(7).normal(0.0, 0.5, n * n)
    conv = (10.0, 10.0)
    h = 1.0 / (n + 1)
    I = np.eye(n)
    Cx, Cy = np.kron(I, upwind_1d(n, conv[0], h)), np.kron(upwind_1d(n, conv[1], h), I)
    K = W.csr_to_dense(W.make_vcdiff(n, theta, conv)) - Cx - Cy  # -div(kappa grad)
    assert np.allclose(K, K.T, rtol=1e-13, atol=1e-9)
    # interior rows sum to zero; a coefficient equals minus its face's kappa / h^2
    kx, ky = W.stencils.vcdiff_faces(n, theta)
    p = np.arange(n * n)
    ix, iy = p % n, p // n
    interior = (ix > 0) & (ix < n - 1) & (iy > 0) & (iy < n - 1)
    assert np.allclose(K[interior].sum(axis=1), 0.0, atol=1e-8 * np.abs(K).max())
    r = 3 + n * 4  # ix = 3, iy = 4
    assert K[r, r - 1] == pytest.approx(-kx[4, 3] / h**2, rel=1e-14)
    assert K[r, r + n] == pytest.approx(-ky[5, 3] / h**2, rel=1e-14)
    # face kappa: the arithmetic mean of the two cells' exp(theta)
    k = np.exp(theta.reshape(n, n))
    assert kx[4, 3] == pytest.approx(0.5 * (k[4, 2] + k[4, 3]), rel=1e-15)


def test_sequence_perturbs_only_the_diagonal():
    A0 = W.make_cd2d(10)
    d = W.diag_perturbation(A0.n)
    assert d.min() >= 0.0 and d.max() < 1.0
    rows = np.repeat(np.arange(A0.n), np.diff(A0.rowptr.astype(np.int64)))
    on = A0.col == rows
    for i, A in enumerate(W.sequence_matrices(A0, 3, 1e-3, d), start=1):
        assert np.array_equal(A.col, A0.col) and np.array_equal(A.rowptr, A0.rowptr)
        assert np.array_equal(A.val[~on], A0.val[~on])
        assert np.allclose(A.val[on] - A0.val[on], i * 1e-3 * d, rtol=0, atol=1e-9)


def test_random_inputs_are_seeded_and_distributed_as_stated():
    N = 200000
    b0, b0again, b1 = W.rhs(N, 0), W.rhs(N, 0), W.rhs(N, 1)
    assert np.array_equal(b0, b0again) and not np.array_equal(b0, b1)
    assert abs(b0.mean()) < 5 / np.sqrt(N) and abs(b0.var() - 1.0) < 0.02
    d = W.diag_perturbation(N)
    assert abs(d.mean() - 0.5) < 5 * np.sqrt(1 / 12 / N)
    th = W.theta_field(64)
    assert th.shape == (4096,) and abs(th.std() - 0.5) < 0.05
    sides_conv = W.batch_systems()
    assert sides_conv == W.batch_systems() and len(sides_conv) == 64
    for side, (cx, cy) in sides_conv:
        assert 32 <= side <= 512 and 1.0 <= cx <= 50.0 and 1.0 <= cy <= 50.0


def test_vcdiff_torch_values_match_numpy_and_differentiate():
    """The torch assembly (differentiable in theta) stores the numpy assembly's
    values in CSR order; its vector-Jacobian product matches central finite
    differences of the numpy assembly."""
    torch = pytest.importorskip("torch")
    from workloads.vcdiff_torch import vcdiff_pattern, vcdiff_values
    n = 9
    theta = np.random.default_rng(11).normal(0.0, 0.5, n * n)
    A = W.make_vcdiff(n, theta)
    rp, col = vcdiff_pattern(n)
    assert np.array_equal(rp, A.rowptr) and np.array_equal(col, A.col)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    vals = vcdiff_values(n, th)
    assert np.allclose(vals.detach().numpy(), A.val, rtol=1e-15, atol=0)
    u = np.random.default_rng(12).standard_normal(A.nnz)
    (g,) = torch.autograd.grad((vals * torch.as_tensor(u)).sum(), th)
    for c in (0, n + 3, n * n // 2, n * n - 1):
        e = np.zeros(n * n)
        e[c] = 1e-6
        fd = (W.make_vcdiff(n, theta + e).val - W.make_vcdiff(n, theta - e).val) @ u / 2e-6
        assert g[c].item() == pytest.approx(fd, rel=1e-6)


def test_dct_draws_are_the_oracle_sketch_draws():
    """The DCT sketch's random signs and rows handed to the library are the ones
    the oracle's SubsampledDCT draws for the same (seed, n, s)."""
    from oracle.sketch import SubsampledDCT
    for seed, n, s in ((231114206, 4096, 120), (7, 250000, 480), (1, 1001, 37)):
        signs, rows = W.dct_draws(seed, n, s)
        S = SubsampledDCT(seed, n, s)
        assert np.array_equal(signs.astype(np.float64), S.signs)
        assert np.array_equal(rows.astype(np.int64), S.rows)
        assert np.all(np.diff(rows) > 0) and rows[0] >= 0 and rows[-1] < n
