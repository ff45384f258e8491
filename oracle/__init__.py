"""Plain, slow FP64 CPU oracle of GMRES-SDR (Burke, Guettel, Soodhalter).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute anything in this package: only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py`` use it.  It shares no code
with the CUDA path (the two sides only share the seeded input generators in
``workloads``); each function cites the part of the paper it follows.

Modules:
  sketch   -- the hash-defined sparse-sign embedding S (Section 3, eq. (sketch)),
              and the subsampled randomised DCT of the paper's experiments
              (Section 6), which the GPU path does not use
  sdr      -- one cycle of Algorithm 1, the restart driver and the sequence
              driver of Section 3.6 (exact and inexact recycling)
  adjoint  -- gradients of L = ||x(theta) - x_t||^2 through A(theta) x = b

Parity unpinned (no closed form to pin them to; the GPU is compared with the
oracle by span only, through principal angles):
  * the harmonic-Ritz selection when |mu_k| and |mu_{k+1}| nearly tie, where
    rounding decides which of the two is kept;
  * the recycle basis U itself, which depends on the choice of basis of the
    selected invariant subspace, while everything downstream depends only on
    its span.
"""
from . import adjoint, sketch, sdr  # noqa: F401
