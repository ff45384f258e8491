"""The five synthetic workloads and their seeded random inputs.

Seeds: sketch 231114206, right-hand sides 1, diagonal perturbations 2, batch
grid sizes 3, log-diffusivity field 4, adjoint target 5.  Every draw uses
numpy's PCG64 through ``default_rng`` with a seed list, so each vector can be
regenerated independently of the order in which others were drawn.
"""
import numpy as np

from .stencils import make_cd2d, make_cd3d, make_vcdiff, perturb_diag

SEEDS = dict(sketch=231114206, b=1, D=2, grid=3, theta=4, target=5)

# Solver parameters per workload (m Krylov columns, k recycled, t window,
# s sketch rows, zeta nonzeros per sketch column).
CONFIGS = {
    "cd2d_64": dict(kind="cd2d", n=64, conv=(10.0, 10.0), systems=1, perturb=0.0,
                    m=50, k=10, t=2, s=120, zeta=8, rel_tol=1e-8),
    "cd3d_128_seq20": dict(kind="cd3d", n=128, conv=(20.0, 10.0, 5.0), systems=20, perturb=1e-3,
                           m=100, k=20, t=2, s=480, zeta=8, rel_tol=1e-8),
    "cd3d_256_seq20_fp32ir": dict(kind="cd3d", n=256, conv=(20.0, 10.0, 5.0), systems=20, perturb=1e-3,
                                  m=80, k=20, t=2, s=400, zeta=8, rel_tol=1e-10),
    "cd2d_batch64": dict(kind="batch", count=64, nmin=32, nmax=512, systems=5, perturb=1e-3,
                         m=40, k=10, t=2, s=100, zeta=8, rel_tol=1e-8),
    "vcdiff_512_adjoint": dict(kind="vcdiff", n=512, conv=(10.0, 10.0), theta_sd=0.5, steps=10,
                               m=60, k=15, t=2, s=300, zeta=8, rel_tol=1e-8),
}


def rhs(N: int, i: int = 0, seed: int = SEEDS["b"]) -> np.ndarray:
    """b^(i) ~ N(0, 1)^N."""
    return np.random.default_rng([seed, i]).standard_normal(N)


def diag_perturbation(N: int, seed: int = SEEDS["D"], tag: int = 0) -> np.ndarray:
    """Diagonal of D ~ U[0, 1]^N used in A^(i) = A0 + i * eps * D."""
    return np.random.default_rng([seed, tag]).random(N)


def sequence_matrices(A0, systems: int, eps: float, dvec=None, first: int = 1):
    """Yield A^(i) = A0 + i * eps * D for i = first .. first + systems - 1."""
    if dvec is None:
        dvec = diag_perturbation(A0.n)
    for i in range(first, first + systems):
        yield perturb_diag(A0, dvec, i * eps) if eps != 0.0 else A0


def base_matrix(cfg: dict):
    if cfg["kind"] == "cd2d":
        return make_cd2d(cfg["n"], cfg["conv"])
    if cfg["kind"] == "cd3d":
        return make_cd3d(cfg["n"], cfg["conv"])
    raise ValueError(cfg["kind"])


def theta_field(n: int, sd: float = 0.5, seed: int = SEEDS["theta"]) -> np.ndarray:
    """Per-cell log-diffusivity theta ~ N(0, sd^2)."""
    return sd * np.random.default_rng([seed, n]).standard_normal(n * n)


def target_field(N: int, seed: int = SEEDS["target"]) -> np.ndarray:
    return np.random.default_rng([seed, N]).standard_normal(N)


def batch_systems(count: int = 64, nmin: int = 32, nmax: int = 512, seed: int = SEEDS["grid"]):
    """Grid sides n ~ U{nmin..nmax} and convection (cx, cy) ~ U[1, 50]^2 per system."""
    rng = np.random.default_rng([seed, count])
    sides = rng.integers(nmin, nmax + 1, size=count)
    conv = rng.uniform(1.0, 50.0, size=(count, 2))
    return [(int(n), (float(c[0]), float(c[1]))) for n, c in zip(sides, conv)]


def dct_draws(seed: int, n: int, s: int):
    """Random draws of the subsampled randomised DCT sketch of the paper's
    experiments (Section 6): n signs +-1 and s distinct rows sorted
    increasingly, from PCG64 seeded [seed, n, s] (signs first, then rows)."""
    g = np.random.default_rng([seed, n, s])
    signs = g.choice(np.array([-1.0, 1.0]), n)
    rows = np.sort(g.choice(n, s, replace=False))
    return signs.astype(np.int8), rows.astype(np.int32)


def vcdiff_problem(n: int, sd: float = 0.5, conv=(10.0, 10.0)):
    theta = theta_field(n, sd)
    return make_vcdiff(n, theta, conv), theta
