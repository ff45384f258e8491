"""The differentiable solve (adjoint form) against the FP64 oracle.

L(theta, b) = ||x - x_t||^2 with A(theta) x = b, the 5-point
variable-coefficient operator (kappa = exp(theta) per cell).  Gradients come
from torch autograd through the library's SDRSolve (forward and transposed
GMRES-SDR solves, each handle with its own recycle space) and the torch
assembly of the stored values.  Bars: the gradient in theta and in b agrees
with the oracle's dense adjoint gradient on the 32 x 32 copy within 1e-8
relative; on the 512 x 512 problem the reverse-mode directional derivative
matches a forward-mode (tangent) solve within 1e-5 and central finite
differences (h = 1e-6) of the GPU loss within their noise.
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as oadj

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEED = 231114206


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2311_14206_gb300 as P
    return P


def make_pair(P, n, rel_tol, m=60, k=15, t=2, s=300):
    from workloads.vcdiff_torch import vcdiff_pattern
    rp, cl = vcdiff_pattern(n)
    rp = torch.as_tensor(rp, device="cuda")
    cl = torch.as_tensor(cl, device="cuda")
    return P.AdjointPair(n * n, rp, cl, m, k, t, s, 8, SEED, rel_tol, max_cycles=400)


def loss_and_grad(P, pair, n, theta, b, x_t):
    from paper_2311_14206_gb300.adjoint import solve
    from workloads.vcdiff_torch import vcdiff_values
    th = torch.as_tensor(theta, device="cuda").requires_grad_(True)
    bt = torch.as_tensor(b, device="cuda").requires_grad_(True)
    xt = torch.as_tensor(x_t, device="cuda")
    x = solve(vcdiff_values(n, th), bt, pair)
    L = torch.sum((x - xt) ** 2)
    L.backward()
    return float(L.detach()), th.grad.cpu().numpy(), bt.grad.cpu().numpy(), x.detach().cpu().numpy()


def gpu_loss(P, pair, n, theta, b, x_t):
    from paper_2311_14206_gb300.adjoint import solve
    from workloads.vcdiff_torch import vcdiff_values
    with torch.no_grad():
        x = solve(vcdiff_values(n, torch.as_tensor(theta, device="cuda")), torch.as_tensor(b, device="cuda"), pair)
        return float(torch.sum((x - torch.as_tensor(x_t, device="cuda")) ** 2))


def inputs(n):
    theta = W.theta_field(n)
    b = W.rhs(n * n, 0)
    x_t = W.target_field(n * n) / (n + 1) ** 2  # on the scale of the solution
    return theta, b, x_t


def test_gradient_matches_dense_oracle_32(P):
    n = 32
    theta, b, x_t = inputs(n)
    pair = make_pair(P, n, 1e-13)
    L, gth, gb, x = loss_and_grad(P, pair, n, theta, b, x_t)
    Lr, xr, lam, dvals, dth = oadj.gradients(n, theta, b, x_t)
    eth = np.max(np.abs(gth - dth)) / np.max(np.abs(dth))
    eb = np.max(np.abs(gb - lam)) / np.max(np.abs(lam))
    print(f"32x32: rel err dL/dtheta {eth:.2e}, dL/db {eb:.2e}, L {abs(L - Lr) / Lr:.2e}")
    assert abs(L - Lr) <= 1e-10 * Lr
    assert eth <= 1e-8
    assert eb <= 1e-8
    # the adjoint handle recycles across calls: a second evaluation at a nearby theta
    L2, gth2, _, _ = loss_and_grad(P, pair, n, theta + 1e-3, b, x_t)
    _, _, _, _, dth2 = oadj.gradients(n, theta + 1e-3, b, x_t)
    assert np.max(np.abs(gth2 - dth2)) / np.max(np.abs(dth2)) <= 1e-8
    assert pair.adj.history()[1][0]["kh"] > 0  # the second adjoint solve started with a recycle space
    pair.close()


def test_gradient_tangent_and_finite_differences_512(P):
    """Reverse mode (the adjoint solve) against forward mode (a tangent solve)
    and against central finite differences of the GPU loss.

    Tangent: A xdot = -(dA/dtheta . v) x, dL/dtheta . v = 2 (x - x_t) . xdot.
    It shares no code with the backward pass beyond the forward solver, so the
    two agree to the solves' accuracy: 1e-5 relative.  The finite-difference
    quotient carries a noise of about kappa(A) tol L / h, and kappa(A) is near
    1e6 on this grid: at tol = 1e-12 and h = 1e-6 it is resolved to about
    1e-2, which is the bar used for it."""
    from workloads.vcdiff_torch import vcdiff_values
    n = 512
    theta, b, x_t = inputs(n)
    pair = make_pair(P, n, 1e-12)
    L, gth, gb, x = loss_and_grad(P, pair, n, theta, b, x_t)
    rng = np.random.default_rng(11)
    v = rng.standard_normal(theta.size)
    g_dir = float(gth @ v)
    # forward mode
    th = torch.as_tensor(theta, device="cuda")
    vals, dvals = torch.func.jvp(lambda t: vcdiff_values(n, t), (th,), (torch.as_tensor(v, device="cuda"),))
    dA = torch.sparse_csr_tensor(pair.rowptr.long(), pair.col.long(), dvals, size=(n * n, n * n))
    xg = torch.as_tensor(x, device="cuda")
    rhs = -(dA @ xg)
    solver = P.Solver(n * n, 60, 15, 2, 300, 8, SEED, 1e-12, max_cycles=400)
    xdot, st, _ = solver.solve(pair.matrix(vals), rhs)
    solver.close()
    t_dir = float(2.0 * (xg - torch.as_tensor(x_t, device="cuda")) @ xdot)
    h = 1e-6
    fd_dir = (gpu_loss(P, pair, n, theta + h * v, b, x_t) - gpu_loss(P, pair, n, theta - h * v, b, x_t)) / (2 * h)
    print(f"512x512: d/dtheta . v adjoint {g_dir:.10e} tangent {t_dir:.10e} (rel {abs(g_dir - t_dir) / abs(t_dir):.2e})"
          f" finite difference {fd_dir:.10e} (rel {abs(g_dir - fd_dir) / abs(fd_dir):.2e})")
    assert st == 0
    assert abs(g_dir - t_dir) <= 1e-5 * abs(t_dir)
    assert abs(g_dir - fd_dir) <= 5e-2 * abs(fd_dir)
    # dL/db = lambda: tangent in b is A xdot = w, d/db . w = 2 (x - x_t) . xdot
    w = rng.standard_normal(b.size)
    solver = P.Solver(n * n, 60, 15, 2, 300, 8, SEED, 1e-12, max_cycles=400)
    xw, st, _ = solver.solve(pair.matrix(vals), torch.as_tensor(w, device="cuda"))
    solver.close()
    tb = float(2.0 * (xg - torch.as_tensor(x_t, device="cuda")) @ xw)
    print(f"  d/db . w adjoint {gb @ w:.10e} tangent {tb:.10e}")
    assert abs(gb @ w - tb) <= 1e-5 * abs(tb)
    pair.close()


def test_transpose_pattern(P):
    """sdr_csr_transpose against the host transpose of the same matrix."""
    A = W.make_vcdiff(17, W.theta_field(17))
    from workloads.stencils import csr_transpose
    T = csr_transpose(A)
    rp = torch.as_tensor(A.rowptr, device="cuda")
    cl = torch.as_tensor(A.col, device="cuda")
    pair = P.AdjointPair(A.n, rp, cl, 20, 4, 2, 40, 8, SEED, 1e-8)
    assert np.array_equal(pair.rowptrT.cpu().numpy(), T.rowptr)
    assert np.array_equal(pair.colT.cpu().numpy(), T.col)
    assert np.array_equal(A.val[pair.perm.cpu().numpy()], T.val)
    pair.close()
