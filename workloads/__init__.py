"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds input generation only: stencil matrices in CSR form,
right-hand sides, diagonal perturbations and coefficient fields.  It contains
none of GMRES-SDR's arithmetic (no sketching, no Krylov steps, no least
squares).  Everything is plain numpy so it runs on any host.
"""
from .stencils import (  # noqa: F401
    CSR,
    make_cd2d,
    make_cd3d,
    make_cd_paper,
    make_vcdiff,
    perturb_diag,
    csr_transpose,
    csr_to_dense,
)
from .configs import (  # noqa: F401
    SEEDS,
    CONFIGS,
    rhs,
    diag_perturbation,
    sequence_matrices,
    theta_field,
    target_field,
    batch_systems,
    dct_draws,
)
