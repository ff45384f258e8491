"""Pins for the oracle's adjoint gradients: central finite differences of the
loss computed by brute force (dense solves), and planted mistakes that the
finite-difference pins must catch."""
import inspect
import types

import numpy as np
import pytest

import workloads as W
from oracle import adjoint
from workloads.stencils import csr_to_dense, make_vcdiff


def problem(n=5, seed=7):
    rng = np.random.default_rng(seed)
    theta = 0.5 * rng.standard_normal(n * n)
    b = rng.standard_normal(n * n)
    x_t = rng.standard_normal(n * n) * 1e-2
    return n, theta, b, x_t


def fd_theta(mod, n, theta, b, x_t, h=1e-6):
    g = np.zeros_like(theta)
    for c in range(theta.size):
        e = np.zeros_like(theta)
        e[c] = h
        g[c] = (mod.loss(n, theta + e, b, x_t) - mod.loss(n, theta - e, b, x_t)) / (2 * h)
    return g


def check_theta(mod):
    n, theta, b, x_t = problem()
    _, _, _, _, dth = mod.gradients(n, theta, b, x_t)
    fd = fd_theta(adjoint, n, theta, b, x_t)
    assert np.max(np.abs(dth - fd)) <= 1e-6 * np.max(np.abs(fd)), np.max(np.abs(dth - fd))


def check_b(mod):
    n, theta, b, x_t = problem(seed=8)
    _, _, lam, _, _ = mod.gradients(n, theta, b, x_t)
    h = 1e-6
    for c in (0, 3, 12, 24):
        e = np.zeros_like(b)
        e[c] = h
        fd = (adjoint.loss(n, theta, b + e, x_t) - adjoint.loss(n, theta, b - e, x_t)) / (2 * h)
        assert abs(lam[c] - fd) <= 1e-6 * max(abs(fd), np.max(np.abs(lam)) * 1e-3)


def check_values(mod):
    """dL/dA_ij against a finite difference of one stored entry of the dense matrix."""
    n, theta, b, x_t = problem(seed=9)
    _, x, _, dvals, _ = mod.gradients(n, theta, b, x_t)
    A = make_vcdiff(n, theta)
    D = csr_to_dense(A)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr.astype(np.int64)))
    h = 1e-7 * np.max(np.abs(D))
    for p in (0, 7, 33, A.nnz - 1):
        i, j = rows[p], A.col[p]
        Dp, Dm = D.copy(), D.copy()
        Dp[i, j] += h
        Dm[i, j] -= h
        Lp = np.sum((np.linalg.solve(Dp, b) - x_t) ** 2)
        Lm = np.sum((np.linalg.solve(Dm, b) - x_t) ** 2)
        fd = (Lp - Lm) / (2 * h)
        assert abs(dvals[p] - fd) <= 1e-5 * max(abs(fd), 1e-12), (p, dvals[p], fd)


PINS = [check_theta, check_b, check_values]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_adjoint_pin(pin):
    pin(adjoint)


def test_grid_32_dense_copy_runs():
    """The 32 x 32 copy used by the GPU gradient test is within the oracle's reach."""
    n = 32
    theta = W.theta_field(n)
    b = W.rhs(n * n, 0)
    x_t = W.target_field(n * n)
    L, x, lam, dvals, dth = adjoint.gradients(n, theta, b, x_t)
    assert np.isfinite(L) and np.all(np.isfinite(dth)) and dvals.size == make_vcdiff(n, theta).nnz


MUTATIONS = [
    ("interior faces without the mean's 1/2", "dth[:, :-1] += 0.5 * k[:, :-1] * q", "dth[:, :-1] += k[:, :-1] * q"),
    ("boundary faces forgotten", "dth[:, 0] += k[:, 0] * bnd[:, 0]", "pass"),
    ("adjoint solved with A instead of A^T", "lam = np.linalg.solve(D.T, 2.0 * r)", "lam = np.linalg.solve(D, 2.0 * r)"),
    ("value gradient with the wrong sign", "dvals = -lam[rows]", "dvals = lam[rows]"),
    ("value gradient with row and column swapped", "dvals = -lam[rows] * x[A.col.astype(np.int64)]",
     "dvals = -lam[A.col.astype(np.int64)] * x[rows]"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_adjoint_mutation_is_caught(name, old, new):
    src = inspect.getsource(adjoint)
    assert src.count(old) >= 1
    mod = types.ModuleType("adjoint_mutant")
    exec(compile(src.replace(old, new, 1), adjoint.__file__ + "<mutant>", "exec"), mod.__dict__)
    caught = False
    for pin in PINS:
        try:
            pin(mod)
        except Exception:  # noqa: BLE001
            caught = True
            break
    assert caught, name
